"""GPU parity of the power spectrum on any survey box (section 3.2, eq.
(Def spec) has no shape restriction): rectangular grids, sides that are not
powers of two (Bluestein transforms), unequal cells and 1D, against the
oracle's estimator with |k| in units of the fundamental of the longest side.
Gates as for the cubic path: mode counts exact, relative 2e-5 per bin
(binary32 transforms) and 1e-10 (binary64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402
from paper_1406_6072_gb300 import workloads as W  # noqa: E402

DEV = torch.device("cuda:0")


def default_kmax(n, cell):
    """The library's default upper edge: the smallest axis Nyquist frequency
    in fundamental units of the longest side (n/2 on a cube)."""
    L = [float(v) * c for v, c in zip(n, cell)]
    lref = max(L)
    return min(0.5 * v * (lref / (float(v) * c)) for v, c in zip(n, cell))


def _run(x, dt, n, cell, bins, F, counts=False, f=None):
    g = cf.make_grid(n, list(cell))
    wsb = cf.cf_power_spectrum_workspace_size(g, F, bins, dt)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    nb = bins.nbins
    pk = torch.empty((F, nb), dtype=torch.float64, device=DEV)
    nm = torch.empty(nb, dtype=torch.int64, device=DEV)
    mean = torch.empty(nb, dtype=torch.float64, device=DEV)
    cov = torch.empty((nb, nb), dtype=torch.float64, device=DEV)
    if counts:
        cf.cf_power_spectrum_counts(x, f, g, F, bins, pk, nm, mean, cov, ws, wsb)
    else:
        cf.cf_power_spectrum(x, dt, g, F, bins, pk, nm, mean, cov, ws, wsb)
    torch.cuda.synchronize()
    return pk.cpu().numpy(), nm.cpu().numpy(), mean.cpu().numpy(), cov.cpu().numpy()


CASES = [((100, 60), (1.0, 1.0), cf.CF_F32, 12, cf.CF_BINS_LINEAR),
         ((100, 60), (1.0, 1.0), cf.CF_F64, 12, cf.CF_BINS_LINEAR),
         ((48, 80, 40), (1.0, 1.0, 1.0), cf.CF_F32, 10, cf.CF_BINS_LINEAR),
         ((48, 80, 40), (1.0, 1.0, 1.0), cf.CF_F64, 8, cf.CF_BINS_LOG),
         ((64, 128), (1.0, 0.5), cf.CF_F64, 16, cf.CF_BINS_LINEAR),     # equal sides, unequal cells
         ((32, 128), (1.0, 1.0), cf.CF_F32, 16, cf.CF_BINS_LINEAR),     # power-of-two rectangle
         ((96, 96), (0.5, 0.5), cf.CF_F32, 20, cf.CF_BINS_LOG),         # non-power-of-two square
         ((24, 40, 12), (1.0, 2.0, 0.5), cf.CF_F32, 6, cf.CF_BINS_LINEAR),
         ((1000,), (1.0,), cf.CF_F64, 25, cf.CF_BINS_LINEAR),           # 1D, long Bluestein line
         ((2048, 3), (1.0, 1.0), cf.CF_F32, 16, cf.CF_BINS_LINEAR),     # longest line, tiny axis
         ((7, 5, 3), (1.0, 1.0, 1.0), cf.CF_F64, 3, cf.CF_BINS_LINEAR)]


@pytest.mark.parametrize("n,cell,dt,nbins,kind", CASES)
def test_any_box_power_spectrum_parity(orc, n, cell, dt, nbins, kind):
    F = 5  # odd: the last field is transformed with a zero partner
    x = W.gaussian_field_values((F,) + n, seed=sum(n), scale=1.1)
    tdt = torch.float32 if dt == cf.CF_F32 else torch.float64
    xt = torch.from_numpy(x).to(tdt).to(DEV)
    kmin = 1.0 if kind == cf.CF_BINS_LOG else 0.0
    bins = cf.make_bins(nbins, kind, kmin, 0.0)
    pk, nm, mean, cov = _run(xt, dt, n, cell, bins, F)
    okind = orc.BINS_LOG if kind == cf.CF_BINS_LOG else orc.BINS_LINEAR
    edges = orc.bin_edges(okind, nbins, kmin, default_kmax(n, cell))
    opk, onm = orc.power_spectrum(xt.double().cpu().numpy(), n, edges, cell=cell)
    assert np.array_equal(nm, onm)
    assert onm.sum() > 0
    tol = 2e-5 if dt == cf.CF_F32 else 1e-10
    assert np.allclose(pk, opk, rtol=tol, atol=tol * opk.max() * 1e-3)
    om, oc = orc.mean_cov(opk)
    assert np.allclose(mean, om, rtol=tol, atol=1e-300)
    assert np.allclose(cov, oc, rtol=10 * tol, atol=10 * tol * np.abs(oc).max())


@pytest.mark.parametrize("n,masked", [((100, 60), True), ((48, 80, 40), False), ((90,), True)])
def test_any_box_count_map_parity(orc, n, masked):
    F = 4
    f = W.survey_mask(n, seed=61) if masked else np.ones(n, dtype=np.float32)
    counts = np.random.default_rng(62).poisson(2.5 * f, size=(F,) + n).astype(np.int32)
    cell = (1.0,) * len(n)
    bins = cf.make_bins(8)
    ct = torch.from_numpy(counts).to(DEV)
    ft = torch.from_numpy(f).to(DEV) if masked else None
    pk, nm, mean, _ = _run(ct, cf.CF_F32, n, cell, bins, F, counts=True, f=ft)
    dg = orc.counts_to_delta(counts.reshape(F, -1), f.ravel().astype(np.float64) if masked else None)
    opk, onm = orc.power_spectrum(dg.reshape((F,) + n), n, orc.bin_edges(0, 8, 0.0, default_kmax(n, cell)))
    assert np.array_equal(nm, onm)
    assert np.allclose(pk, opk, rtol=2e-5, atol=1e-7 * opk.max())
    assert np.allclose(mean, opk.mean(0), rtol=2e-5)


def test_sampled_fields_of_a_non_power_of_two_survey(orc):
    """End to end on a 100 x 60 survey: the sampler (embedded in the next
    power of two) and the spectrum of its fields, both against the oracle."""
    n, R, seed = (100, 60), 3, 71
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, seed, 0, R, cf.CF_F32, fields, ws, wsb)
    torch.cuda.synchronize()
    M = [int(2 ** np.ceil(np.log2(2 * v))) for v in n]
    o = orc.embed(list(n), orc.XI_GAUSSIAN, 1.0, 3.0, M=M)
    ref = orc.sample(n, o["sqrt_lambda"], seed, 0, R, 1)
    got = fields.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    bins = cf.make_bins(10)
    pk, nm, _, _ = _run(fields, cf.CF_F32, n, (1.0, 1.0), bins, 2 * R)
    opk, onm = orc.power_spectrum(got.reshape((2 * R,) + n), n, orc.bin_edges(0, 10, 0.0, default_kmax(n, (1, 1))))
    assert np.array_equal(nm, onm)
    assert np.allclose(pk, opk, rtol=2e-5, atol=1e-7 * opk.max())
    emb.close()
