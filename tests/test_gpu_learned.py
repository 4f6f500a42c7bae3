"""The learned preconditioner on the GPU against the oracle's network: inference,
loss and Wirtinger gradients, gauge equivariance, training, the flexible GCR
solver with and without the network, and the network as the TSM's LP map."""
import numpy as np
import pytest

import synth
from oracle import loops, network, noise
from oracle import operator as op

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


def _ctx(dl, dims, links, kappa, amu):
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
    dl.dl_set_params(ctx, kappa, amu)
    return ctx


def _shapes(n_layers, c):
    return [(1 if l == 0 else c, 1 if l == n_layers - 1 else c) for l in range(n_layers)]


def _to_oracle(flat, n_layers, c):
    """[9][4][C_out][C_in] per layer -> the oracle's {W0 [o,i,2], Wf/Wb [4,o,i,4]} dicts."""
    out, k = [], 0
    for ci, co in _shapes(n_layers, c):
        w = flat[k:k + 36 * co * ci].astype(np.complex128).reshape(9, 4, co, ci)
        k += 36 * co * ci
        out.append({"W0": np.moveaxis(w[0, :2], 0, -1),
                    "Wf": np.stack([np.moveaxis(w[1 + 2 * mu], 0, -1) for mu in range(4)]),
                    "Wb": np.stack([np.moveaxis(w[2 + 2 * mu], 0, -1) for mu in range(4)])})
    return out


def _from_oracle(ws):
    parts = []
    for w in ws:
        co, ci = w["W0"].shape[:2]
        f = np.zeros((9, 4, co, ci), dtype=np.complex128)
        f[0, :2] = np.moveaxis(w["W0"], -1, 0)
        for mu in range(4):
            f[1 + 2 * mu] = np.moveaxis(w["Wf"][mu], -1, 0)
            f[2 + 2 * mu] = np.moveaxis(w["Wb"][mu], -1, 0)
        parts.append(f.ravel())
    return np.concatenate(parts)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("act,tol", [("f32", 2e-6), ("bf16", 3e-2)])
@pytest.mark.parametrize("n_layers,c", [(4, 16), (3, 5)])
def test_forward_matches_oracle(dl, act, tol, n_layers, c):
    dims = (4, 4, 4, 8)
    links = synth.gauge_links(dims, 0.4, 311)
    w = synth.network_weights(n_layers, c, 57, scale=0.6, identity=0.5)
    eta = np.stack([noise.z4_noise(dims, 12, r) for r in range(2)])
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_F32 if act == "f32" else dl.DL_BF16)
        dl.dl_nn_set_weights(nn, w)
        assert np.array_equal(dl.dl_nn_get_weights(nn), w)
        out = torch.zeros(eta.size, dtype=torch.complex128, device="cuda")
        dl.dl_nn_apply(nn, 2, _dev(eta), out)
        got = out.cpu().numpy().reshape(eta.shape)
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ws = _to_oracle(w, n_layers, c)
    for r in range(2):
        ref, _ = network.forward(links, ws, eta[r])
        assert np.abs(got[r] - ref).max() <= tol * np.abs(ref).max(), r


def test_tensor_core_forward_matches_cuda_core_forward(dl):
    """bfloat16 network, 16 channels on an 8^4 lattice (several 128-site CTAs): the
    tcgen05 channel mixing against the CUDA-core forward and against the oracle."""
    dims = (8, 8, 8, 8)
    links = synth.gauge_links(dims, 0.4, 317)
    w = synth.network_weights(4, 16, 65, scale=0.6, identity=0.5)
    eta = np.stack([noise.z4_noise(dims, 15, r) for r in range(2)])
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    outs = {}
    try:
        nn = dl.dl_nn_create(ctx, 4, 16, dl.DL_BF16)
        dl.dl_nn_set_weights(nn, w)
        for tc in (1, 0):
            dl.dl_nn_set_tensor_cores(nn, tc)
            out = torch.zeros(eta.size, dtype=torch.complex128, device="cuda")
            dl.dl_nn_apply(nn, 2, _dev(eta), out)
            outs[tc] = out.cpu().numpy().reshape(eta.shape)
        dl.dl_nn_destroy(nn)
        nn32 = dl.dl_nn_create(ctx, 4, 16, dl.DL_F32)
        with pytest.raises(dl.DLError):
            dl.dl_nn_set_tensor_cores(nn32, 1)
        dl.dl_nn_destroy(nn32)
    finally:
        dl.dl_destroy(ctx)
    ws = _to_oracle(w, 4, 16)
    for r in range(2):
        ref, _ = network.forward(links, ws, eta[r])
        sc = np.abs(ref).max()
        assert np.abs(outs[1][r] - ref).max() <= 3e-2 * sc, r
        assert np.abs(outs[1][r] - outs[0][r]).max() <= 3e-2 * sc, r


def test_tensor_core_adjoint_matches_oracle(dl):
    """bfloat16 network, 16 channels on an 8^4 lattice: N^+ y on the tensor cores (the
    adjoint layers as forward layers of conjugate-transposed, hop-swapped weights) against
    the CUDA-core input-gradient kernels and the oracle's layer adjoints; and
    <N x, y> = <x, N^+ y> within the bfloat16 rounding of both sides."""
    dims = (8, 8, 8, 8)
    n_layers, c = 4, 16
    links = synth.gauge_links(dims, 0.4, 318)
    w = synth.network_weights(n_layers, c, 66, scale=0.6, identity=0.5)
    y = synth.gaussian_spinors(dims, 2, 67)
    x = synth.gaussian_spinors(dims, 2, 68)
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    outs = {}
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_BF16)
        dl.dl_nn_set_weights(nn, w)
        for tc in (1, 0):
            dl.dl_nn_set_tensor_cores(nn, tc)
            out = torch.zeros(y.size, dtype=torch.complex128, device="cuda")
            dl.dl_nn_apply_adjoint(nn, 2, _dev(y), out)
            outs[tc] = out.cpu().numpy().reshape(y.shape)
        dl.dl_nn_set_tensor_cores(nn, 1)
        nx = torch.zeros(x.size, dtype=torch.complex128, device="cuda")
        dl.dl_nn_apply(nn, 2, _dev(x), nx)
        nx = nx.cpu().numpy().reshape(x.shape)
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ws = _to_oracle(w, n_layers, c)
    for r in range(2):
        g = y[r:r + 1]
        for li in range(n_layers - 1, -1, -1):
            ci = 1 if li == 0 else c
            x0 = np.zeros((ci,) + dims[::-1] + (4, 3), dtype=np.complex128)
            _, g = network.layer_backward(links, ws[li], x0, g)
        sc = np.abs(g).max()
        assert np.abs(outs[1][r] - g[0]).max() <= 3e-2 * sc, r
        assert np.abs(outs[1][r] - outs[0][r]).max() <= 3e-2 * sc, r
        lhs, rhs = np.vdot(nx[r], y[r]), np.vdot(x[r], outs[1][r])
        assert abs(lhs - rhs) <= 2e-2 * np.linalg.norm(nx[r]) * np.linalg.norm(y[r]), r


def test_adjoint_matches_oracle(dl):
    """N^+ y from the input-gradient kernels against the oracle's layer adjoints (FP32)."""
    dims = (4, 4, 4, 4)
    n_layers, c = 4, 16
    links = synth.gauge_links(dims, 0.4, 316)
    w = synth.network_weights(n_layers, c, 63, scale=0.6, identity=0.5)
    y = synth.gaussian_spinors(dims, 1, 64)
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_F32)
        dl.dl_nn_set_weights(nn, w)
        out = torch.zeros(y.size, dtype=torch.complex128, device="cuda")
        dl.dl_nn_apply_adjoint(nn, 1, _dev(y), out)
        got = out.cpu().numpy().reshape(y.shape)
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ws = _to_oracle(w, n_layers, c)
    g = y  # [1, ...] one channel at the output
    for li in range(n_layers - 1, -1, -1):
        ci = 1 if li == 0 else c
        x0 = np.zeros((ci,) + dims[::-1] + (4, 3), dtype=np.complex128)  # the input only enters gw
        _, g = network.layer_backward(links, ws[li], x0, g)
    assert np.abs(got - g).max() <= 2e-6 * np.abs(g).max()


def test_loss_and_gradients_match_oracle(dl):
    """Loss and every weight gradient (2 dL/d conj W) of three pairs, FP32 activations."""
    dims = (4, 4, 2, 4)
    n_layers, c = 3, 4
    links = synth.gauge_links(dims, 0.4, 312)
    w = synth.network_weights(n_layers, c, 58, scale=0.8, identity=0.7)
    eta = np.stack([noise.z4_noise(dims, 13, r) for r in range(3)])
    s = synth.gaussian_spinors(dims, 3, 59)
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_F32)
        dl.dl_nn_set_weights(nn, w)
        loss, grad = dl.dl_nn_loss_grad(nn, 3, _dev(eta), _dev(s))
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ref_loss, ref_grads = network.loss_and_grads(links, _to_oracle(w, n_layers, c), list(zip(eta, s)))
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    ref = _from_oracle(ref_grads)
    used = np.ones(ref.size, dtype=bool)
    k = 0
    for ci, co in _shapes(n_layers, c):
        m = np.ones((9, 4, co, ci), dtype=bool)
        m[0, 2:] = False
        used[k:k + m.size] = m.ravel()
        k += m.size
    assert np.all(grad[~used] == 0)
    assert np.abs(grad - ref).max() <= 2e-5 * np.abs(ref).max()


def test_tensor_core_gradients_match_oracle(dl):
    """bfloat16 network, 16 channels, on 6x6x2x4 (4.5 tiles of 32 sites per parity): the
    weight gradients of the tensor-core kernel (the sites as the reduction dimension of the
    products) against the CUDA-core kernel and the oracle, layer by layer, within the
    bfloat16 rounding of the activations; unused weight slots stay zero."""
    dims = (6, 6, 2, 4)
    n_layers, c = 3, 16
    links = synth.gauge_links(dims, 0.4, 319)
    w = synth.network_weights(n_layers, c, 69, scale=0.6, identity=0.5)
    eta = np.stack([noise.z4_noise(dims, 17, r) for r in range(2)])
    s = synth.gaussian_spinors(dims, 2, 70)
    ctx = _ctx(dl, dims, links, 0.16, 0.01)
    got = {}
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_BF16)
        dl.dl_nn_set_weights(nn, w)
        for tc in (1, 0):
            dl.dl_nn_set_tensor_cores(nn, tc)
            got[tc] = dl.dl_nn_loss_grad(nn, 2, _dev(eta), _dev(s))
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ref_loss, ref_grads = network.loss_and_grads(links, _to_oracle(w, n_layers, c), list(zip(eta, s)))
    ref = _from_oracle(ref_grads)
    for tc in (1, 0):
        assert abs(got[tc][0] - ref_loss) <= 3e-2 * ref_loss, tc
    k = 0
    for ci, co in _shapes(n_layers, c):
        sl = slice(k, k + 36 * co * ci)
        k += 36 * co * ci
        sc = np.abs(ref[sl]).max()
        assert np.abs(got[1][1][sl] - ref[sl]).max() <= 5e-2 * sc, (ci, co)
        assert np.abs(got[1][1][sl] - got[0][1][sl]).max() <= 5e-2 * sc, (ci, co)
        unused = np.zeros((9, 4, co, ci), dtype=bool)
        unused[0, 2:] = True
        assert np.all(got[1][1][sl][unused.ravel()] == 0)


def test_residual_loss_and_gradients_match_oracle(dl):
    """The residual loss |M_u N eta - eta|^2 / |eta|^2 of three sources and every weight
    gradient, FP32 activations, against the oracle (M applied in FP32 on the GPU)."""
    dims = (4, 4, 2, 4)
    n_layers, c = 3, 4
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.4, 315)
    w = synth.network_weights(n_layers, c, 60, scale=0.8, identity=0.7)
    eta = np.stack([noise.z4_noise(dims, 14, r) for r in range(3)])
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        nn = dl.dl_nn_create(ctx, n_layers, c, dl.DL_F32)
        dl.dl_nn_set_weights(nn, w)
        loss, grad = dl.dl_nn_loss_grad_residual(nn, 3, _dev(eta))
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    ref_loss, ref_grads = network.residual_loss_and_grads(links, _to_oracle(w, n_layers, c), list(eta), kappa, amu)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    ref = _from_oracle(ref_grads)
    assert np.abs(grad - ref).max() <= 2e-5 * np.abs(ref).max()


def test_gauge_equivariance_on_gpu(dl):
    """N[U^G](G eta) = G N[U](eta) for a random SU(3) gauge transformation G."""
    dims = (4, 4, 4, 4)
    links = synth.gauge_links(dims, 0.4, 313)
    g = synth.gauge_transform_field(dims, 314)
    lg = np.empty_like(links)
    for mu in range(4):
        gf = np.roll(g, -1, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])
        lg[..., mu, :, :] = g @ links[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    w = synth.network_weights(4, 16, 60, scale=0.6, identity=0.5)
    eta = noise.z4_noise(dims, 14, 0)
    outs = []
    for lk, e in ((links, eta), (lg, op.colour(g, eta))):
        ctx = _ctx(dl, dims, lk, 0.16, 0.01)
        try:
            nn = dl.dl_nn_create(ctx, 4, 16, dl.DL_F32)
            dl.dl_nn_set_weights(nn, w)
            out = torch.zeros(e.size, dtype=torch.complex128, device="cuda")
            dl.dl_nn_apply(nn, 1, _dev(e), out)
            outs.append(out.cpu().numpy().reshape(e.shape))
            dl.dl_nn_destroy(nn)
        finally:
            dl.dl_destroy(ctx)
    ref = op.colour(g, outs[0])
    assert np.abs(outs[1] - ref).max() <= 3e-6 * np.abs(ref).max()


@pytest.mark.parametrize("normal", [0, 1])
def test_fgcr_without_network_matches_dense(dl, normal):
    """Flexible GCR with the identity preconditioner (on M, or on M^+ M) reaches 1e-10;
    solution vs dense LU."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    eta = np.stack([noise.z4_noise(dims, 2000, r) for r in range(3)])
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        sol = torch.zeros(eta.size, dtype=torch.complex128, device="cuda")
        prm = dl.dl_fgcr_params(tol=1e-10, max_iter=5000, restart=16, inner_tol=1e-5, flavour=1, normal=normal)
        st, stats = dl.dl_fgcr_solve(ctx, None, prm, 3, _dev(eta), sol)
        assert st == 0
        got = sol.cpu().numpy().reshape(eta.shape)
    finally:
        dl.dl_destroy(ctx)
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    for r in range(3):
        assert stats.true_resid[r] <= 1e-10
        s = (minv @ eta[r].ravel()).reshape(eta[r].shape)
        assert np.linalg.norm(got[r] - s) <= 1e-8 * np.linalg.norm(s)
        res = op.apply_m(links, got[r], kappa, amu, 1) - eta[r]
        assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(eta[r])


@pytest.fixture(scope="module")
def trained(dl):
    """An 8^4 lattice, 48 (noise, FP64 solution) pairs from the plain solver, and a
    4-layer, 16-channel BF16 network trained on them with Adam."""
    dims = (8, 8, 8, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 315)
    V = int(np.prod(dims))
    n = 48
    ctx = _ctx(dl, dims, links, kappa, amu)
    eta = torch.zeros(n * V * 12, dtype=torch.complex128, device="cuda")
    sol = torch.zeros_like(eta)
    prm = dl.dl_solve_params(tol=1e-10, max_iter=50000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.01, flavour=1,
                             chunk=0)
    for b in range(0, n, 16):
        dl.dl_noise_z4(ctx, 2024, b, 16, eta[b * V * 12:(b + 16) * V * 12])
        st, _ = dl.dl_solve(ctx, eta[b * V * 12:(b + 16) * V * 12], sol[b * V * 12:(b + 16) * V * 12], 16,
                            dl.DL_C128, prm)
        assert st == 0
    nn = dl.dl_nn_create(ctx, 4, 16, dl.DL_BF16)
    w0 = synth.network_weights(4, 16, 61)
    dl.dl_nn_set_weights(nn, w0)
    tp = dl.dl_nn_train_params(steps=400, batch=4, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=7)
    hist = dl.dl_nn_train(nn, tp, n, eta, sol)
    yield dict(dl=dl, ctx=ctx, nn=nn, links=links, dims=dims, kappa=kappa, amu=amu, hist=hist, w0=w0, V=V)
    dl.dl_nn_destroy(nn)
    dl.dl_destroy(ctx)


def test_training_reduces_loss(trained):
    h = trained["hist"]
    assert np.all(np.isfinite(h))
    assert h[-20:].mean() < 0.7 * h[:20].mean(), (h[:20].mean(), h[-20:].mean())


@pytest.mark.parametrize("normal", [0, 1])
def test_trained_network_preconditions_fgcr(trained, normal):
    """Fresh noise: FGCR to 1e-10 with the trained network needs fewer iterations than
    without it (same restart length; on M the unpreconditioned solve may stagnate, on
    M^+ M both converge); the solutions satisfy M s = eta to 1e-10 (oracle)."""
    dl, ctx, nn, V = trained["dl"], trained["ctx"], trained["nn"], trained["V"]
    n = 4
    eta = torch.zeros(n * V * 12, dtype=torch.complex128, device="cuda")
    dl.dl_noise_z4(ctx, 4048, 0, n, eta)
    prm = dl.dl_fgcr_params(tol=1e-10, max_iter=3000, restart=32, inner_tol=1e-4, flavour=1, normal=normal)
    out = {}
    for name, net in (("plain", None), ("net", nn)):
        sol = torch.zeros_like(eta)
        st, stats = dl.dl_fgcr_solve(ctx, net, prm, n, eta, sol)
        assert st == 0 or (name == "plain" and not normal and st == dl.DL_NOT_CONVERGED)
        out[name] = (np.array(stats.iters[:n]), sol.cpu().numpy())
    assert out["net"][0].mean() < 0.8 * out["plain"][0].mean(), (out["net"][0], out["plain"][0])
    e = eta.cpu().numpy().reshape((n,) + trained["dims"][::-1] + (4, 3))
    s = out["net"][1].reshape(e.shape)
    for r in range(n):
        res = op.apply_m(trained["links"], s[r], trained["kappa"], trained["amu"], 1) - e[r]
        assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(e[r])


def test_tsm_with_learned_lp_map(dl):
    """Eq. estiTSM with the network as the LP map: the HP terms use dense-exact
    solutions, the LP terms the oracle network's output with the same weights."""
    dims = (4, 4, 4, 4)
    kappa, amu = 0.16, 0.01
    links = synth.gauge_links(dims, 0.3, 1000)
    n_hp, n_lp = 3, 5
    w = synth.network_weights(3, 8, 62, scale=0.5, identity=0.9)
    ctx = _ctx(dl, dims, links, kappa, amu)
    try:
        nn = dl.dl_nn_create(ctx, 3, 8, dl.DL_F32)
        dl.dl_nn_set_weights(nn, w)
        prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-11, tol_lp=1e-2, prec_hp_lo=dl.DL_F64,
                               prec_lp_lo=dl.DL_F32, delta_hp=0.1, block=4, seed=2000, p2max=0, with_deriv=0, hpe=0,
                               max_iter=50000, chunk=8, lp_net=nn["h"])
        out = np.zeros((2, dims[3], 1, 1, 4, 4), dtype=np.complex128)
        st, info = dl.dl_tsm_run(ctx, prm, out)
        assert st == 0 and info.iters_lp == 0
        dl.dl_nn_destroy(nn)
    finally:
        dl.dl_destroy(ctx)
    minv = np.linalg.inv(op.dense_matrix(links, kappa, amu, 1))
    ws = _to_oracle(w, 3, 8)

    def functional(est, e, s):
        """The loop functional the TSM applies to any map's output: for the generalised
        estimator D_W s is taken as eta - 2i kappa amu g5 s (equal for the exact s,
        and what the GPU evaluates for every map)."""
        if est == "one_end":
            xi, phi = loops.g5(s), s
        else:
            xi, phi = loops.g5(s), loops.g5(e - 2j * kappa * amu * loops.g5(s))
        return loops.prefactor(est, kappa, amu) * loops.bilinear(xi, phi).sum(axis=(1, 2, 3))

    for k, est in enumerate(("one_end", "gen_one_end")):
        fh, fl = [], []
        for r in range(n_hp + n_lp):
            e = noise.z4_noise(dims, 2000, r)
            s_lp, _ = network.forward(links, ws, e)
            f = lambda s: functional(est, e, s)
            fl.append(f(s_lp))
            if r < n_hp:
                fh.append(f((minv @ e.ravel()).reshape(e.shape)))
        ref = loops.tsm_estimate(fh, fl[:n_hp], fl[n_hp:])
        assert np.abs(out[k, :, 0, 0] - ref).max() <= 1e-5 * np.abs(ref).max(), est
