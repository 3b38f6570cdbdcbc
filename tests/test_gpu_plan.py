"""GPU tests of captured plans (cf_plan_*): every replay draws the next R
realizations; its fields and counts are bit-identical to the eager calls
(cf_sample_lp) on the same realization range, and its power spectra equal
cf_power_spectrum / cf_power_spectrum_counts up to the order of the atomic
bin sums."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _eager(emb, n, seed, r0, R, sigma2, nbar, lp_seed, bins, nbins):
    F = 2 * R
    grid = cf.make_grid(n)
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    cf.cf_sample_lp(emb, seed, r0, R, cf.CF_F32, fields, cf.make_lp(sigma2, nbar, counts, lp_seed), ws, wsb)
    pkb = cf.cf_power_spectrum_workspace_size(grid, F, bins, cf.CF_F32)
    pkws = torch.empty(pkb, dtype=torch.uint8, device=DEV)
    pk = torch.empty((F, nbins), dtype=torch.float64, device=DEV)
    pkc = torch.empty_like(pk)
    nm = torch.empty(nbins, dtype=torch.int64, device=DEV)
    mean = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cov = torch.empty((nbins, nbins), dtype=torch.float64, device=DEV)
    cf.cf_power_spectrum(fields, cf.CF_F32, grid, F, bins, pk, nm, mean, cov, pkws, pkb)
    cf.cf_power_spectrum_counts(counts, None, grid, F, bins, pkc, nm, None, None, pkws, pkb)
    torch.cuda.synchronize()
    return fields, counts, pk, pkc, mean, cov


@pytest.mark.parametrize("n,kind,scale", [((64, 64), cf.CF_XI_GAUSSIAN, 4.0), ((32, 32, 32), cf.CF_XI_EXPONENTIAL, 3.0)])
def test_plan_replays_match_eager_calls(n, kind, scale):
    R, nbins, seed, lp_seed, sigma2, nbar = 3, 12, 77, 78, 0.7, 2.5
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(kind, 0.7, scale), cf.CF_EMBED_CLAMP)
    bins = cf.make_bins(nbins)
    F = 2 * R
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    pk = torch.empty((F, nbins), dtype=torch.float64, device=DEV)
    pkc = torch.empty_like(pk)
    nm = torch.empty(nbins, dtype=torch.int64, device=DEV)
    mean = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cov = torch.empty((nbins, nbins), dtype=torch.float64, device=DEV)
    lp = cf.make_lp(sigma2, nbar, counts, lp_seed)
    plan = cf.Plan(emb, seed, 10, R, fields, lp=lp, bins=bins, pk=pk, nmodes=nm, mean=mean, cov=cov, pk_counts=pkc)
    for k in range(3):  # launches draw [10, 13), [13, 16), [16, 19)
        plan.launch()
        torch.cuda.synchronize()
        ef, ec, epk, epkc, emean, ecov = _eager(emb, n, seed, 10 + R * k, R, sigma2, nbar, lp_seed, bins, nbins)
        assert torch.equal(fields, ef), k
        assert torch.equal(counts, ec), k
        # bin sums use binary32 partial sums and atomic additions: the spectra agree
        # to rounding order (other realizations would differ at order one).  The
        # covariance's small entries are differences of products of spectra
        # that agree to about 1e-7, so they are compared against its largest
        # entry.
        for a, b in ((pk, epk), (pkc, epkc), (mean, emean)):
            assert torch.allclose(a, b, rtol=1e-6, atol=1e-9 * float(b.abs().max())), k
        assert torch.allclose(cov, ecov, rtol=1e-5, atol=1e-6 * float(ecov.abs().max())), k
    plan.seek(13)
    plan.launch()
    torch.cuda.synchronize()
    ef, ec, _, _, _, _ = _eager(emb, n, seed, 13, R, sigma2, nbar, lp_seed, bins, nbins)
    assert torch.equal(fields, ef) and torch.equal(counts, ec)
    plan.close()
    emb.close()


def test_plan_fields_only_and_errors():
    n = (32, 64)
    R = 2
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    plan = cf.Plan(emb, 5, 0, R, fields)
    plan.launch()
    torch.cuda.synchronize()
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    ref = torch.empty_like(fields)
    cf.cf_sample(emb, 5, 0, R, cf.CF_F32, ref, ws, wsb)
    torch.cuda.synchronize()
    assert torch.equal(fields, ref)
    plan.close()
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    f = torch.ones(n, dtype=torch.float32, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.Plan(emb, 5, 0, R, fields, lp=cf.make_lp(0.5, 1.0, counts, 3, f=f))
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    emb.close()
