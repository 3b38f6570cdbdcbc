"""Full-size parity: the workloads at their real sizes, run exactly as
bench.py runs them (FieldPipeline: embed, fused sample + lognormal/Poisson in
chunks of up to 1 GiB of intermediate, both power spectra), checked on realizations sampled across
the batch against the oracle, which computes them one by one.  Tolerances as
in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402
from paper_1406_6072_gb300 import workloads as W  # noqa: E402
from paper_1406_6072_gb300.pipeline import FieldPipeline  # noqa: E402

DEV = torch.device("cuda:0")


def _check_realization(orc, wl, o_emb, fields, counts, pk, pkg, r, r0):
    n = wl.n
    ref = orc.sample(n, o_emb["sqrt_lambda"], wl.seed, r0 + r, 1, 1)[0]
    got = fields[r].double().cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, (r, err)
    G = got.reshape(2, -1)
    _, oc, margin = orc.lognormal_poisson(G, wl.sigma2, wl.nbar, seed=wl.seed + 1000, field0=2 * (r0 + r))
    c = counts[r].cpu().numpy().reshape(2, -1)
    bad = (c != oc) & (margin >= 1e-6)
    assert not bad.any(), (r, int(bad.sum()))
    assert (margin < 1e-6).mean() < 1e-3
    edges = orc.bin_edges(orc.BINS_LINEAR, wl.nbins, 0.0, n[0] / 2)
    opk, _ = orc.power_spectrum(got, n, edges)
    gpk = pk[2 * r:2 * r + 2].cpu().numpy()
    assert np.allclose(gpk, opk, rtol=2e-5, atol=1e-9 * opk.max()), r
    dg = orc.counts_to_delta(c, None).reshape((2,) + tuple(n))
    opkg, _ = orc.power_spectrum(dg, n, edges)
    assert np.allclose(pkg[2 * r:2 * r + 2].cpu().numpy(), opkg, rtol=2e-5, atol=1e-9 * opkg.max()), r


@pytest.mark.parametrize("name,sampled", [("cauchy2d_n512_f32", (0, 37, 63)), ("exp3d_n128", (5,))])
def test_workload_at_full_size(orc, name, sampled):
    wl = W.CONFIGS[name]
    pipe = FieldPipeline(wl, "cuda:0")
    r0 = 3 * wl.R
    pipe.step(r0=r0)
    torch.cuda.synchronize()
    o_emb = orc.embed(list(wl.n), wl.xi_kind, wl.amp, wl.scale, wl.beta, clamp=wl.clamp)
    rep, orep = pipe.emb.report, o_emb["report"]
    assert rep["n_negative"] == orep["n_negative"] and rep["clamped"] == orep["clamped"]
    lam = torch.empty(wl.m, dtype=torch.float64, device="cuda:0")
    cf.cf_embedding_lambda(pipe.emb, lam)
    torch.cuda.synchronize()
    lmax = o_emb["lambda"].max()
    assert np.max(np.abs(lam.cpu().numpy() - o_emb["lambda"])) <= 1e-12 * lmax
    if wl.clamp:
        assert rep["cov_error"] == pytest.approx(orep["cov_error"], rel=1e-6)
    for r in sampled:
        _check_realization(orc, wl, o_emb, pipe.fields, pipe.counts, pipe.pk, pipe.pkg, r, r0)
    # mean and covariance over all fields of the batch
    pk = pipe.pk.cpu().numpy()
    mean, cov = orc.mean_cov(pk)
    assert np.allclose(pipe.mean.cpu().numpy(), mean, rtol=1e-12)
    assert np.allclose(pipe.cov.cpu().numpy(), cov, rtol=1e-9, atol=1e-12 * np.abs(cov).max())
    nm = pipe.nmodes.cpu().numpy()
    assert nm.sum() > 0 and np.all(nm >= 0)
    pipe.close()


@pytest.fixture(scope="module")
def cauchy_n512(orc):
    """The 512^2 generalised-Cauchy workload's embedding (not PSD, clamped)
    from the oracle: row, eigenvalues and report."""
    wl = W.CONFIGS["cauchy2d_n512_f32"]
    return wl, orc.embed(list(wl.n), wl.xi_kind, wl.amp, wl.scale, wl.beta, clamp=True)


def _check_clamp_report(rep, orep):
    # section 2, eq. (condition): the clamped spectrum's realised covariance
    # error is the method's statement of how far the sample is from exact
    assert rep["clamped"] == 1 and orep["clamped"] == 1
    assert rep["n_negative"] == orep["n_negative"]
    assert abs(rep["n_zeroed"] - orep["n_zeroed"]) <= max(2, orep["n_zeroed"] // 100)
    assert rep["neg_mass"] == pytest.approx(orep["neg_mass"], rel=1e-9)
    assert rep["cov_error"] == pytest.approx(orep["cov_error"], rel=1e-6)


@pytest.mark.parametrize("on_device", [False, True])
def test_tabulated_row_clamp_report_at_full_size(cauchy_n512, on_device):
    """The general (complex-transform) embedding path with a tabulated first
    row at 1024^2: the grid-stride passes wrap many times here, so any
    overlap between the clamped spectrum and its transform buffer shows."""
    wl, o = cauchy_n512
    tab = torch.from_numpy(np.ascontiguousarray(o["c"]))
    if on_device:
        tab = tab.to(DEV)
    emb = cf.cf_embed(cf.make_grid(wl.n), cf.make_xi(cf.CF_XI_TABLE, table=tab), cf.CF_EMBED_CLAMP)
    lam = torch.empty(o["lambda"].shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    assert np.max(np.abs(lam.cpu().numpy() - o["lambda"])) <= 1e-12 * o["lambda"].max()
    _check_clamp_report(emb.report, o["report"])
    emb.close()


def test_explicit_lambda_clamp_report_at_full_size(cauchy_n512):
    """cf_embed_from_lambda at 1024^2 with the oracle's (non-PSD) eigenvalues."""
    wl, o = cauchy_n512
    lam = torch.from_numpy(np.ascontiguousarray(o["lambda"])).to(DEV)
    emb = cf.cf_embed_from_lambda(cf.make_grid(wl.n), lam, cf.CF_EMBED_CLAMP)
    torch.cuda.synchronize()
    _check_clamp_report(emb.report, o["report"])
    emb.close()
