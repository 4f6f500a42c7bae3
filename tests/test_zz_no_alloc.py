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


def test_noalloc_matches_dl_apply_twice(dl):
    dims = (4, 6, 4, 8)
    kappa, amu = 0.161, 0.0055
    links = synth.gauge_links(dims, 0.4, 91)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    try:
        dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
        dl.dl_set_params(ctx, kappa, amu)
        cases = [(dl.DL_OP_M, dl.DL_F64, 3), (dl.DL_OP_MHAT, dl.DL_F32, 5), (dl.DL_OP_RECON, dl.DL_F64, 4),
                 (dl.DL_OP_BH, dl.DL_F16, 8)]
        for call in range(2):
            for k, (op, prec, n) in enumerate(cases):
                x = torch.from_numpy(synth.gaussian_spinors(dims, n, 92 + 10 * call + k)).cuda()
                a = torch.from_numpy(synth.gaussian_spinors(dims, n, 93 + 10 * call + k)).cuda()
                ref = torch.empty_like(x)
                got = torch.full_like(x, float("nan"))
                dl.dl_apply(ctx, op, prec, 1, n, x, a, ref, dl.DL_C128)
                dl.dl_apply_noalloc(ctx, op, prec, 1, n, x, a, got, dl.DL_C128)
                torch.cuda.synchronize()
                r, g = ref.cpu().numpy(), got.cpu().numpy()
                tol = {dl.DL_F64: 1e-13, dl.DL_F32: 2e-6, dl.DL_F16: 3e-4}[prec]
                assert np.isfinite(g).all()
                assert np.abs(g - r).max() <= tol * np.abs(r).max(), (call, op, prec)
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
