"""GPU tests of the counts-in-cells kernels (section 3.4) against the oracle:
the histogram bit for bit (integer work), its mean and covariance over maps,
the Poisson-lognormal mixture prediction (trapezoid rule on the GPU, adaptive
quadrature in the oracle: two quadratures of one integral) and the A* transform
of eq. (As) (Newton on the GPU, bisection in the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402
from paper_1406_6072_gb300 import workloads as W  # noqa: E402

DEV = torch.device("cuda:0")


def _counts(orc, shape, F, sigma2, nbar, masked, seed):
    cells = int(np.prod(shape))
    f = W.survey_mask(shape, seed=seed).ravel() if masked else None
    G = W.gaussian_field_values((F, cells), seed=seed + 1, scale=np.sqrt(sigma2))
    _, counts, _ = orc.lognormal_poisson(G, sigma2, nbar, f=f, seed=seed + 2)
    return counts.astype(np.int32), f


@pytest.mark.parametrize("shape,F,nbins,masked", [((64, 64), 6, 42, True), ((37, 29), 3, 8, False),
                                                 ((128, 128), 2, 1024, True)])
def test_histogram_bit_exact(orc, shape, F, nbins, masked):
    counts, f = _counts(orc, shape, F, 0.8, 4.0, masked, 40)
    cells = counts.shape[1]
    c = torch.from_numpy(counts).to(DEV)
    fd = torch.from_numpy(f).to(DEV) if f is not None else None
    hist = torch.empty((F, nbins), dtype=torch.float64, device=DEV)
    mean = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cov = torch.empty((nbins, nbins), dtype=torch.float64, device=DEV)
    cf.cf_cic_histogram(c, cells, F, fd, nbins, hist, mean, cov)
    torch.cuda.synchronize()
    ref = orc.cic_histogram(counts, f, nbins)
    assert np.array_equal(hist.cpu().numpy(), ref)
    om, oc = orc.mean_cov(ref)
    assert np.allclose(mean.cpu().numpy(), om, rtol=1e-13, atol=0)
    assert np.allclose(cov.cpu().numpy(), oc, rtol=1e-11, atol=1e-12 * max(1.0, np.abs(oc).max()))


@pytest.mark.parametrize("sigma2,nbar,masked,nbins", [(0.13, 9.68, True, 42), (0.8, 2.0, False, 64),
                                                      (1.0, 0.5, True, 16)])
def test_prediction_matches_oracle(orc, sigma2, nbar, masked, nbins):
    shape = (64, 64)
    f = W.survey_mask(shape, seed=41).ravel() if masked else None
    fd = torch.from_numpy(f).to(DEV) if f is not None else None
    cells = int(np.prod(shape))
    pred = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cf.cf_cic_prediction(sigma2, nbar, fd, cells, nbins, pred)
    torch.cuda.synchronize()
    ref = orc.cic_prediction(sigma2, nbar, f if f is not None else np.ones(cells), nbins)
    got = pred.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-8, atol=1e-10 * cells), np.max(np.abs(got - ref) / ref)


def test_astar_matches_oracle(orc):
    counts, f = _counts(orc, (64, 64), 4, 0.13, 9.68, True, 50)
    counts[0, :50] = np.arange(50) * 40  # large counts too
    cells = counts.shape[1]
    out = torch.empty(counts.shape, dtype=torch.float32, device=DEV)
    cf.cf_astar(torch.from_numpy(counts).to(DEV), torch.from_numpy(f).to(DEV), cells, 4, 9.68, 0.13, out)
    torch.cuda.synchronize()
    ref = orc.astar(counts, f, 9.68, 0.13)
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(got[:, f == 0] == 0)
    assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) < 2e-7


def test_cic_argument_errors():
    c = torch.zeros((1, 16), dtype=torch.int32, device=DEV)
    h = torch.empty((1, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.cf_cic_histogram(c, 16, 1, None, 2000, h)
    assert ei.value.status == cf.CF_ERR_ARG
    with pytest.raises(cf.CfError) as ei:
        cf.cf_cic_prediction(0.5, 1.0, None, 16, 65, h)
    assert ei.value.status == cf.CF_ERR_ARG
    with pytest.raises(cf.CfError) as ei:
        cf.cf_astar(c, None, 16, 1, 1.0, 0.0, h)
    assert ei.value.status == cf.CF_ERR_ARG


@pytest.mark.parametrize("nbins,F", [(16, 400), (64, 2000), (300, 4000)])
def test_cumulative_information_matches_oracle(orc, nbins, F):
    rng = np.random.default_rng(nbins)
    pk = rng.gamma(3.0, 1.0, size=(F, nbins)) * np.linspace(1.0, 0.2, nbins)[None, :]
    pk[:, 1:] += 0.3 * pk[:, :-1]  # correlated neighbouring bins
    pk[:, 3] = 0.0                 # a bin without modes
    mean, cov = orc.mean_cov(pk)
    ref = orc.cumulative_information(mean, cov)
    m = torch.from_numpy(mean).to(DEV)
    c = torch.from_numpy(cov).to(DEV)
    out = torch.empty(nbins, dtype=torch.float64, device=DEV)
    wsb = cf.cumulative_information_workspace_size(nbins)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    cf.cf_cumulative_information(m, c, nbins, out, ws, wsb)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-9)


def test_cumulative_information_singular_is_nan(orc):
    nbins, F = 12, 6  # fewer fields than bins: the covariance is singular
    pk = np.random.default_rng(1).gamma(3.0, 1.0, size=(F, nbins))
    mean, cov = orc.mean_cov(pk)
    out = torch.empty(nbins, dtype=torch.float64, device=DEV)
    wsb = cf.cumulative_information_workspace_size(nbins)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    cf.cf_cumulative_information(torch.from_numpy(mean).to(DEV), torch.from_numpy(cov).to(DEV), nbins, out, ws, wsb)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(np.isfinite(o[:F - 1])) and np.isnan(o[-1])
