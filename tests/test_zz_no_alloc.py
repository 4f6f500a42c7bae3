"""The allocation-free operator entry point against dl_apply.

dl_apply_noalloc serves callers that cannot allocate device memory when they
apply an operator (a framework allocator owning the device memory, a
latency-critical loop); it must return what dl_apply returns.  Two calls in a
row check that the shared fixed scratch carries nothing from one call into the
next.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_2256_gb300 as m
    m.lib()
    return m


OPS = ["M", "MDAG", "HOP", "MHAT", "MHAT_DAG", "PREP", "RECON", "BH"]


def test_noalloc_matches_dl_apply_twice(dl):
    """Every operator in every storage precision, each called twice in a row with fresh
    inputs: the result equals dl_apply's within the operator tolerances of these tests."""
    dims = (4, 6, 4, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 91)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, kappa, amu)
        tols = {dl.DL_F64: 1e-13, dl.DL_F32: 2e-6, dl.DL_F16: 3e-4}
        for call in range(2):
            for k, name in enumerate(OPS):
                for j, prec in enumerate((dl.DL_F64, dl.DL_F32, dl.DL_F16)):
                    n = 1 + (3 * k + j + call) % 8
                    seed = 1000 * call + 10 * k + j
                    x = torch.from_numpy(synth.gaussian_spinors(dims, n, 92 + seed)).cuda()
                    a = torch.from_numpy(synth.gaussian_spinors(dims, n, 93 + seed)).cuda()
                    ref = torch.empty_like(x)
                    got = torch.full_like(x, float("nan"))
                    op = getattr(dl, "DL_OP_" + name)
                    dl.dl_apply(ctx, op, prec, 1, n, x, a, ref, dl.DL_C128)
                    dl.dl_apply_noalloc(ctx, op, prec, 1, n, x, a, got, dl.DL_C128)
                    torch.cuda.synchronize()
                    r, g = ref.cpu().numpy(), got.cpu().numpy()
                    assert np.isfinite(g).all(), (call, name, prec)
                    assert np.abs(g - r).max() <= tols[prec] * np.abs(r).max(), (call, name, prec)
    finally:
        dl.dl_destroy(ctx)


def _noalloc_need(vh, n, site_bytes, scales):
    """The header's size rule: 7 x ceil256(V/2 x npad x site bytes) [+ 7 x ceil256 of the
    4-byte scales of the 16-bit format], npad = n rounded up to a power of two."""
    npad = 1
    while npad < n:
        npad *= 2
    c256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    return 7 * (c256(vh * npad * site_bytes) + (c256(vh * npad * 4) if scales else 0))


@pytest.mark.parametrize("t_ext,fits", [(24, True), (26, False)])
def test_noalloc_size_limit(dl, t_ext, fits):
    """Just below and just above the 64 MiB limit (FP64, one right-hand side on
    16^3 x T): the first runs and matches dl_apply, the second is rejected."""
    dims = (16, 16, 16, t_ext)
    vh = 16 ** 3 * t_ext // 2
    need = _noalloc_need(vh, 1, 192, False)
    assert (need <= 64 << 20) == fits and abs(need - (64 << 20)) < 0.1 * (64 << 20)
    links = synth.unit_links(dims)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, 0.12, 0.01)
        x = torch.from_numpy(synth.gaussian_spinors(dims, 1, 95)).cuda()
        got = torch.full_like(x, float("nan"))
        if fits:
            ref = torch.empty_like(x)
            dl.dl_apply(ctx, dl.DL_OP_M, dl.DL_F64, 1, 1, x, None, ref, dl.DL_C128)
            dl.dl_apply_noalloc(ctx, dl.DL_OP_M, dl.DL_F64, 1, 1, x, None, got, dl.DL_C128)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max()
        else:
            with pytest.raises(dl.DLError) as e:
                dl.dl_apply_noalloc(ctx, dl.DL_OP_M, dl.DL_F64, 1, 1, x, None, got, dl.DL_C128)
            assert e.value.status == dl.DL_ERR_ARG
            assert "fixed scratch" in dl.dl_last_error(ctx)
    finally:
        dl.dl_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(dl):
    dims = (16, 16, 16, 16)
    links = synth.unit_links(dims)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, 0.12, 0.01)
        x = torch.zeros((32, 16 ** 4 * 12), dtype=torch.complex128, device="cuda")
        with pytest.raises(dl.DLError) as e:
            dl.dl_apply_noalloc(ctx, dl.DL_OP_M, dl.DL_F64, 1, 32, x, None, x.clone(), dl.DL_C128)
        assert e.value.status == dl.DL_ERR_ARG
        assert "fixed scratch" in dl.dl_last_error(ctx)
    finally:
        dl.dl_destroy(ctx)
