"""The live stencil statistics (dl_profile, dl_profile_stencils) that the benchmark's
roofline is computed from: launches counted per class including the solver's CUDA-graph
replays, durations from CUDA events."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F32, B16 = 1, 2  # storage slots of dl_profile_stencils
PLAIN, AUX, AUXN, CGU = 0, 1, 2, 3


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("n", [4, 16])
def test_stencil_statistics_of_a_fixed_solve(dl, n):
    """Eight CG iterations (16-bit Krylov vectors, FP32 accumulation, no reliable
    updates; four iterations per graph launch): each of the four 16-bit CG stencil classes
    runs exactly 8 times, and is timed by the one sampled iteration; the FP32 launches
    outside the graph (source preparation, the two residual recomputations at the end,
    reconstruction, true residual) are all counted and timed."""
    dims = (4, 4, 4, 8)
    links = synth.gauge_links(dims, 0.4, 401)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, 0.161, 0.0055)
        eta = torch.empty((n,) + dims[::-1] + (4, 3), dtype=torch.complex64, device="cuda")
        dl.dl_noise_z4(ctx, 402, 0, n, eta, dl.DL_C64)
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=1e-30, max_iter=8, prec_hi=dl.DL_F32, prec_lo=dl.DL_F16, delta=0.0, flavour=1,
                                 chunk=4)
        dl.dl_solve(ctx, eta, sol, n, dl.DL_C64, prm)  # graphs and workspaces
        dl.dl_profile(ctx, 1)
        dl.dl_solve(ctx, eta, sol, n, dl.DL_C64, prm)
        st = dl.dl_profile_stencils()
        st2 = dl.dl_profile_stencils()  # reading twice does not count twice
        dl.dl_profile(ctx, 0)
    finally:
        dl.dl_destroy(ctx)
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    for e, d in ((PLAIN, 0), (AUXN, 0), (PLAIN, 1), (CGU, 1)):
        n_l, n_t, ms, items = st[B16, e, d]
        assert n_l == 8, (e, d, n_l)
        assert n_t == 1 and ms > 0 and items == vh * n, (e, d, n_t, ms, items)
    assert st[B16, AUX].sum() == 0 and st[B16, CGU, 0].sum() == 0
    f32 = st[F32]
    assert f32[:, :, 0].sum() > 0 and np.array_equal(f32[:, :, 0], f32[:, :, 1])  # every FP32 launch timed
    assert (f32[:, :, 2] >= 0).all() and f32[:, :, 2].sum() > 0
    assert np.array_equal(st, st2)
    assert st[0].sum() == 0 and st[3].sum() == 0  # no double-float or IEEE FP64 launches
