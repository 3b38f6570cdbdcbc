"""GPU tests of cf_sample_spectra: the sampler's last pass fused with the
first axis of the fields' power spectrum.  Fields and counts are the ones of
cf_sample / cf_sample_lp bit for bit (same kernels up to the epilogue); the
spectra, mean and covariance equal cf_power_spectrum on those fields up to
rounding (the two axes are transformed in the other order) and the oracle's
spectra of the same fields within the binary32 gate."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _run(emb, n, R, nbins, lp_args, fused):
    seed, r0 = 61, 5
    bins = cf.make_bins(nbins)
    grid = cf.make_grid(n)
    F = 2 * R
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.full((R, 2) + n, -9, dtype=torch.int32, device=DEV) if lp_args else None
    lp = cf.make_lp(*lp_args[:2], counts, lp_args[2]) if lp_args else None
    pk = torch.empty((F, nbins), dtype=torch.float64, device=DEV)
    nm = torch.empty(nbins, dtype=torch.int64, device=DEV)
    mean = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cov = torch.empty((nbins, nbins), dtype=torch.float64, device=DEV)
    if fused:
        pkb = cf.cf_sample_spectra_workspace_size(emb, R, bins)
        pkws = torch.empty(pkb, dtype=torch.uint8, device=DEV)
        cf.cf_sample_spectra(emb, seed, r0, R, fields, lp, bins, pk, nm, mean, cov, ws, wsb, pkws, pkb)
    else:
        if lp is not None:
            cf.cf_sample_lp(emb, seed, r0, R, cf.CF_F32, fields, lp, ws, wsb)
        else:
            cf.cf_sample(emb, seed, r0, R, cf.CF_F32, fields, ws, wsb)
        pkb = cf.cf_power_spectrum_workspace_size(grid, F, bins, cf.CF_F32)
        pkws = torch.empty(pkb, dtype=torch.uint8, device=DEV)
        cf.cf_power_spectrum(fields, cf.CF_F32, grid, F, bins, pk, nm, mean, cov, pkws, pkb)
    torch.cuda.synchronize()
    return fields, counts, pk, nm, mean, cov


@pytest.mark.parametrize("n,R,nbins,lp_args", [((128, 128), 3, 16, (0.8, 2.0, 7)), ((512, 512), 4, 64, (0.8, 2.0, 8)),
                                               ((256, 256), 5, 33, None), ((1024, 1024), 2, 40, (0.5, 9.7, 9))])
def test_fused_spectra_match_separate_calls(orc, n, R, nbins, lp_args):
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 6.0, 0.4), cf.CF_EMBED_CLAMP)
    a = _run(emb, n, R, nbins, lp_args, fused=True)
    b = _run(emb, n, R, nbins, lp_args, fused=False)
    assert torch.equal(a[0], b[0])
    if lp_args:
        assert torch.equal(a[1], b[1])
    assert torch.equal(a[3], b[3])
    for x, y in ((a[2], b[2]), (a[4], b[4])):
        assert torch.allclose(x, y, rtol=2e-5, atol=0), float(((x - y).abs() / y.abs()).max())
    assert torch.allclose(a[5], b[5], rtol=1e-4, atol=1e-6 * float(b[5].abs().max()))
    # against the oracle's spectra of the same fields
    g = a[0].double().cpu().numpy().reshape((2 * R,) + n)
    edges = orc.bin_edges(orc.BINS_LINEAR, nbins, 0.0, n[0] / 2)
    opk, onm = orc.power_spectrum(g, n, edges)
    assert np.array_equal(a[3].cpu().numpy(), onm)
    got = a[2].cpu().numpy()
    sel = onm > 0
    assert np.max(np.abs(got[:, sel] - opk[:, sel]) / np.abs(opk[:, sel])) < 2e-5
    emb.close()


def test_fused_spectra_refusals():
    bins = cf.make_bins(8)
    for n in ((64, 64), (128, 256), (128, 128, 128)):
        emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
        with pytest.raises(cf.CfError) as ei:
            cf.cf_sample_spectra_workspace_size(emb, 2, bins)
        assert ei.value.status == cf.CF_ERR_UNSUPPORTED
        emb.close()
    emb = cf.cf_embed(cf.make_grid((128, 128)), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    f = torch.empty((1, 2, 128, 128), dtype=torch.float32, device=DEV)
    pk = torch.empty((2, 8), dtype=torch.float64, device=DEV)
    nm = torch.empty(8, dtype=torch.int64, device=DEV)
    wsb = cf.cf_sample_workspace_size(emb, 1, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    small = torch.empty(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.cf_sample_spectra(emb, 1, 0, 1, f, None, bins, pk, nm, None, None, ws, wsb, small, 64)
    assert ei.value.status == cf.CF_ERR_NOMEM
    emb.close()


def test_fused_spectra_with_chunked_workspace():
    """A sampler workspace of two realizations (several chunks, ragged last)
    gives the same fields as one chunk, and the same spectra up to the order
    of their atomic bin sums."""
    n, R, nbins = (256, 256), 5, 24
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 5.0))
    bins = cf.make_bins(nbins)
    pkb = cf.cf_sample_spectra_workspace_size(emb, R, bins)
    out = []
    for wsr in (R, 2):
        wsb = cf.cf_sample_workspace_size(emb, wsr, cf.CF_F32)
        ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
        fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
        pk = torch.empty((2 * R, nbins), dtype=torch.float64, device=DEV)
        nm = torch.empty(nbins, dtype=torch.int64, device=DEV)
        pkws = torch.empty(pkb, dtype=torch.uint8, device=DEV)
        cf.cf_sample_spectra(emb, 3, 11, R, fields, None, bins, pk, nm, None, None, ws, wsb, pkws, pkb)
        torch.cuda.synchronize()
        out.append((fields, pk))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.allclose(out[0][1], out[1][1], rtol=2e-5, atol=0)
    emb.close()
