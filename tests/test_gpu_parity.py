"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerances:
  * noise: bit-exact;
  * eigenvalues: |lambda_gpu - lambda_oracle| <= 1e-12 lambda_max;
  * fields: relative L2 <= 1e-10 (binary64), <= 1e-5 (binary32);
  * counts: bit-exact except cells whose intensity lies within relative 1e-6
    of an inverse-CDF boundary (counted, must be rare);
  * power spectra: relative 1e-10 (binary64), 2e-5 (binary32) per bin; mode
    counts exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402
from paper_1406_6072_gb300 import workloads as W  # noqa: E402

DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def gpu_noise(seed, r0, R, ncells, m_last, dt):
    t = torch.empty((R, ncells, 2), dtype=torch.float32 if dt == cf.CF_F32 else torch.float64, device=DEV)
    cf.cf_draw_noise(seed, r0, R, ncells, m_last, dt, t)
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1], t


@pytest.mark.parametrize("seed,r0,R,ncells,m_last", [(1, 0, 3, 4096, 64), (0xDEADBEEF12345678, 2**32 - 4, 4, 1024, 1024),
                                                      (7, 123, 2, 24, 2), (2, 5, 1, 8192, 4096)])
def test_noise_bit_exact(orc, seed, r0, R, ncells, m_last):
    for dt, odt in ((cf.CF_F64, 0), (cf.CF_F32, 1)):
        got, t = gpu_noise(seed, r0, R, ncells, m_last, dt)
        ref = orc.draw_noise(seed, r0, R, ncells, m_last, odt)
        if dt == cf.CF_F32:
            g32 = t.cpu().numpy().view(np.uint32)
            r32 = np.stack([ref.real, ref.imag], -1).astype(np.float32).view(np.uint32)
            assert np.array_equal(g32, r32), "binary32 noise differs in %d words" % int((g32 != r32).sum())
        else:
            g64 = t.cpu().numpy().view(np.uint64)
            r64 = np.stack([ref.real, ref.imag], -1).view(np.uint64)
            assert np.array_equal(g64, r64), "binary64 noise differs in %d words" % int((g64 != r64).sum())


EMBED_CASES = [
    ((64,), 0, 1.0, 3.0, 0.0, False),
    ((64, 64), 0, 1.0, 4.0, 0.0, False),          # Gaussian s=4 (the 2D binary64 workload)
    ((16, 32), 2, 1.3, 1.5, 0.0, False),          # rectangular
    ((8, 16, 4), 2, 0.7, 0.8, 0.0, False),        # 3D rectangular
    ((64, 64), 1, 0.8, 8.0, 0.4, True),           # generalised Cauchy, not PSD -> clamped
    ((1, 1), 0, 1.0, 1.0, 0.0, False),            # degenerate 2x2 embedding
    ((2048,), 1, 0.8, 16.0, 0.4, True),           # longest line
]


@pytest.mark.parametrize("n,kind,amp,scale,beta,clamp", EMBED_CASES)
def test_embedding_parity(orc, n, kind, amp, scale, beta, clamp):
    o = orc.embed(list(n), kind, amp, scale, beta, clamp=clamp)
    g = cf.make_grid(n)
    emb = cf.cf_embed(g, cf.make_xi(kind, amp, scale, beta), cf.CF_EMBED_CLAMP if clamp else 0)
    M = tuple(2 * v for v in n)
    lam = torch.empty(M, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    s = torch.empty(M, dtype=torch.float64, device=DEV)
    cf.cf_embedding_sqrt_lambda(emb, s)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    lmax = o["lambda"].max()
    assert np.max(np.abs(lam - o["lambda"])) <= 1e-12 * lmax
    rep, orep = emb.report, o["report"]
    assert rep["lambda_max"] == pytest.approx(orep["lambda_max"], rel=1e-12)
    assert abs(rep["lambda_min"] - orep["lambda_min"]) <= 1e-12 * lmax
    assert rep["n_negative"] == orep["n_negative"]
    assert rep["clamped"] == orep["clamped"]
    assert abs(rep["n_zeroed"] - orep["n_zeroed"]) <= max(2, orep["n_zeroed"] // 100)
    if clamp:
        assert rep["cov_error"] == pytest.approx(orep["cov_error"], rel=1e-6, abs=1e-13)
        assert rep["neg_mass"] == pytest.approx(orep["neg_mass"], rel=1e-9)
    # sqrt(lambda+) agrees where both sides took the same threshold decision;
    # squared, the difference is bounded by the eigenvalue tolerance
    same = (lam > rep["tau"]) == (o["lambda"] > orep["tau"])
    sg = s.cpu().numpy()[same]
    so = o["sqrt_lambda"][same]
    assert np.max(np.abs(sg * sg - so * so)) <= 1e-12 * lmax
    emb.close()


@pytest.mark.parametrize("on_device", [False, True])
def test_embedding_from_table(orc, on_device):
    """A tabulated first row (the general, not necessarily even, path): here the
    row of the generalised-Cauchy family plus an odd perturbation."""
    n = (16, 32)
    c = orc.embed_row(list(n), 1, 0.8, 3.0, 0.4)
    c = c + 1e-3 * np.sin(2 * np.pi * np.arange(c.shape[1]) / c.shape[1])[None, :]
    tab = torch.from_numpy(np.ascontiguousarray(c))
    if on_device:
        tab = tab.to(DEV)
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_TABLE, table=tab), cf.CF_EMBED_CLAMP)
    lam = torch.empty(c.shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    ref = np.real(orc.fft_nd(c.astype(np.complex128), -1))
    assert np.max(np.abs(lam.cpu().numpy() - ref)) <= 1e-12 * np.abs(ref).max()
    _, _, orep = orc.psd(list(n), c, ref, clamp=True)
    assert emb.report["n_negative"] == orep["n_negative"]
    if orep["clamped"]:
        assert emb.report["cov_error"] == pytest.approx(orep["cov_error"], rel=1e-6, abs=1e-13)
    emb.close()


@pytest.mark.parametrize("table,on_device", [(False, False), (True, False), (True, True)])
def test_embedding_log1p_input(orc, table, on_device):
    """CF_EMBED_LOG1P (eq. (Lncov)): the embedded covariance is ln(1 + xi),
    parametric and tabulated xi."""
    n = (32, 64)
    o = orc.embed(list(n), 1, 0.14, 4.0, 0.4, clamp=True, log1p=True)
    if table:
        tab = torch.from_numpy(np.ascontiguousarray(orc.embed_row(list(n), 1, 0.14, 4.0, 0.4)))
        if on_device:
            tab = tab.to(DEV)
        xi = cf.make_xi(cf.CF_XI_TABLE, table=tab)
    else:
        xi = cf.make_xi(1, 0.14, 4.0, 0.4)
    emb = cf.cf_embed(cf.make_grid(n), xi, cf.CF_EMBED_CLAMP | cf.CF_EMBED_LOG1P)
    lam = torch.empty(o["lambda"].shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    lmax = o["lambda"].max()
    assert np.max(np.abs(lam.cpu().numpy() - o["lambda"])) <= 1e-12 * lmax
    assert emb.report["n_negative"] == o["report"]["n_negative"]
    emb.close()
    with pytest.raises(cf.CfError) as ei:
        cf.cf_embed(cf.make_grid(n), cf.make_xi(1, -1.5, 4.0, 0.4), cf.CF_EMBED_LOG1P)
    assert ei.value.status == cf.CF_ERR_ARG


def test_not_psd_is_reported(orc):
    g = cf.make_grid((64, 64))
    with pytest.raises(cf.CfError) as ei:
        cf.cf_embed(g, cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 8.0, 0.4), 0)
    assert ei.value.status == cf.CF_ERR_NOT_PSD
    o = orc.embed([64, 64], 1, 0.8, 8.0, 0.4)
    assert ei.value.report["n_negative"] == o["report"]["n_negative"] > 0


SAMPLE_CASES = [
    ((64, 64), 0, 4.0, 3, 5),      # 2D
    ((16, 128), 2, 1.5, 2, 3),     # rectangular, long rows
    ((8, 8), 0, 0.9, 4, 7),        # tiny: one CTA of mostly idle rows
    ((256,), 2, 5.0, 3, 2),        # 1D
    ((8, 16, 32), 2, 1.0, 2, 3),   # 3D rectangular
    ((32, 32, 32), 2, 1.5, 2, 2),  # 3D cube
    ((2, 4), 2, 0.5, 3, 1),        # very small
]


def _fields(emb, seed, r0, R, dt, n, ws_real=None):
    ws_bytes = cf.cf_sample_workspace_size(emb, R, dt)
    if ws_real is not None:
        ws_bytes = cf.cf_sample_workspace_size(emb, ws_real, dt)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + tuple(n), dtype=torch.float32 if dt == cf.CF_F32 else torch.float64, device=DEV)
    cf.cf_sample(emb, seed, r0, R, dt, out, ws, ws_bytes)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,kind,scale,R,r0", SAMPLE_CASES)
def test_sample_component_parity(orc, n, kind, scale, R, r0):
    """GPU sampler fed the oracle's lambda: identical threshold decisions."""
    o = orc.embed(list(n), kind, 1.0, scale, 0.4, clamp=True)
    g = cf.make_grid(n)
    lam = torch.from_numpy(o["lambda"]).to(DEV)
    emb = cf.cf_embed_from_lambda(g, lam, cf.CF_EMBED_CLAMP)
    seed = 0x1234567890 + R
    for dt, odt, tol in ((cf.CF_F64, 0, 1e-10), (cf.CF_F32, 1, 1e-5)):
        got = _fields(emb, seed, r0, R, dt, n).double().cpu().numpy()
        ref = orc.sample(n, o["sqrt_lambda"], seed, r0, R, odt)
        assert rel_l2(got, ref) <= tol, (dt, rel_l2(got, ref))
    emb.close()


def test_sample_chunked_workspace_matches_unchunked(orc):
    n = (32, 64)
    g = cf.make_grid(n)
    emb = cf.cf_embed(g, cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 2.0))
    full = _fields(emb, 5, 9, 7, cf.CF_F32, n)
    chunked = _fields(emb, 5, 9, 7, cf.CF_F32, n, ws_real=2)   # chunks of 2, ragged last chunk
    assert torch.equal(full, chunked)
    part = _fields(emb, 5, 12, 2, cf.CF_F32, n)                 # realizations 12, 13 alone
    assert torch.equal(full[3:5], part)
    with pytest.raises(cf.CfError) as ei:
        out = torch.empty((2, 2) + n, device=DEV)
        cf.cf_sample(emb, 5, 0, 2, cf.CF_F32, out, torch.empty(8, dtype=torch.uint8, device=DEV), 8)
    assert ei.value.status == cf.CF_ERR_NOMEM
    out = torch.zeros((1, 2) + n, device=DEV)
    cf.cf_sample(emb, 5, 0, 0, cf.CF_F32, out, None, 0)        # R = 0 is a no-op
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0
    with pytest.raises(cf.CfError):
        cf.cf_sample(emb, 5, 2**32 - 1, 2, cf.CF_F32, out, None, 0)
    emb.close()


def test_end_to_end_binary64_workload(orc):
    """The 2D 64x64 binary64 workload: embed + sample on the GPU against the
    oracle's embed + sample (threshold-decision differences reported)."""
    wl = W.CONFIGS["gauss2d_n64_f64"]
    o = orc.embed(list(wl.n), wl.xi_kind, wl.amp, wl.scale, wl.beta)
    emb = cf.cf_embed(cf.make_grid(wl.n), cf.make_xi(wl.xi_kind, wl.amp, wl.scale, wl.beta), 0)
    lam = torch.empty(wl.m, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    differing = int(((lam.cpu().numpy() > emb.report["tau"]) != (o["lambda"] > o["report"]["tau"])).sum())
    got = _fields(emb, wl.seed, 0, wl.R, cf.CF_F64, wl.n).cpu().numpy()
    ref = orc.sample(wl.n, o["sqrt_lambda"], wl.seed, 0, wl.R, 0)
    err = rel_l2(got, ref)
    print("binary64 workload: rel L2 %.3e, threshold decisions differing: %d" % (err, differing))
    assert err <= 1e-10
    emb.close()


def _lp_check(orc, G, counts, delta, sigma2, nbar, f, seed, field0, flag_limit=1e-3):
    Gd = np.asarray(G, dtype=np.float64).reshape(G.shape[0], -1)
    od, oc, margin = orc.lognormal_poisson(Gd, sigma2, nbar, f=f, seed=seed, field0=field0)
    c = np.asarray(counts).reshape(oc.shape)
    flagged = margin < 1e-6
    bad = (c != oc) & ~flagged
    assert not bad.any(), "%d counts differ outside the boundary band" % int(bad.sum())
    assert flagged.mean() < flag_limit
    if delta is not None:
        d = np.asarray(delta, dtype=np.float64).reshape(od.shape)
        assert np.max(np.abs(d - od) / (1 + np.abs(od))) < 2e-6
    return int(flagged.sum()), int((c != oc).sum())


@pytest.mark.parametrize("dt", [cf.CF_F32, cf.CF_F64])
@pytest.mark.parametrize("nbar,sigma2,masked,field0", [(2.0, 0.8, False, 0), (0.5, 1.0, True, 3), (40.0, 1.5, True, 10),
                                                      (1e-3, 0.2, False, 1)])
def test_lognormal_poisson_parity(orc, dt, nbar, sigma2, masked, field0):
    cells, nf = 4096, 6
    G = W.gaussian_field_values((nf, cells), seed=31, scale=np.sqrt(sigma2))
    f = W.survey_mask((64, 64), seed=32).ravel() if masked else None
    tdt = torch.float32 if dt == cf.CF_F32 else torch.float64
    Gt = torch.from_numpy(G).to(tdt).to(DEV)
    ft = torch.from_numpy(f).to(DEV) if f is not None else None
    counts = torch.empty((nf, cells), dtype=torch.int32, device=DEV)
    delta = torch.empty((nf, cells), dtype=torch.float32, device=DEV)
    cf.cf_lognormal_poisson(Gt, dt, cells, nf, sigma2, nbar, ft, 77, field0, delta, counts)
    torch.cuda.synchronize()
    fl, nd = _lp_check(orc, Gt.double().cpu().numpy(), counts.cpu().numpy(), delta.cpu().numpy(), sigma2, nbar,
                       None if f is None else f.astype(np.float64), 77, field0)
    print("flagged %d, differing %d" % (fl, nd))


def test_fused_sample_lp_parity(orc):
    n = (64, 64)
    R, seed, pseed = 4, 21, 22
    g = cf.make_grid(n)
    emb = cf.cf_embed(g, cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 4.0, 0.4), cf.CF_EMBED_CLAMP)
    plain = _fields(emb, seed, 2, R, cf.CF_F32, n)
    f = W.survey_mask(n, seed=23)
    ft = torch.from_numpy(f).to(DEV)
    ws_bytes = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=DEV)
    fields = torch.empty_like(plain)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    delta = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    lp = cf.make_lp(0.8, 2.0, counts, pseed, f=ft, delta_out=delta)
    cf.cf_sample_lp(emb, seed, 2, R, cf.CF_F32, fields, lp, ws, ws_bytes)
    torch.cuda.synchronize()
    assert torch.equal(fields, plain)
    _lp_check(orc, fields.double().cpu().numpy().reshape(2 * R, -1), counts.cpu().numpy().reshape(2 * R, -1),
              delta.cpu().numpy().reshape(2 * R, -1), 0.8, 2.0, f.ravel().astype(np.float64), pseed, field0=4)
    # the standalone kernel on the same fields gives the same counts
    c2 = torch.empty_like(counts)
    cf.cf_lognormal_poisson(fields, cf.CF_F32, n[0] * n[1], 2 * R, 0.8, 2.0, ft, pseed, 4, None, c2)
    torch.cuda.synchronize()
    assert torch.equal(c2, counts)
    emb.close()


@pytest.mark.parametrize("n,nbar,sigma2", [((128, 128), 40.0, 1.5), ((64, 64, 32), 9.68, 0.8), ((1024,), 2.0, 0.8)])
def test_deferred_binary64_decisions(orc, n, nbar, sigma2):
    """Counts the binary32 walk leaves undecided go to a list in the workspace
    and are decided by a second kernel; with a workspace too small for the
    list they are decided in place.  Both give the same counts, which match
    the oracle (up to flagged boundary cells)."""
    R, seed, pseed = 3, 51, 52
    g = cf.make_grid(n)
    emb = cf.cf_embed(g, cf.make_xi(cf.CF_XI_GAUSSIAN, sigma2, 3.0))
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = {}
    M = [2 * v for v in n]
    one = 8 * int(np.prod(M[:-1])) * n[-1] if len(n) == 2 else None
    sizes = {"list": cf.cf_sample_workspace_size(emb, R, cf.CF_F32)}
    if len(n) == 2:
        sizes["in_place"] = one  # one realization's intermediates and no room for the list
    else:
        sizes["in_place"] = 0 if len(n) == 1 else None
    for name, wsb in sizes.items():
        if wsb is None:
            continue
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
        c = torch.full((R, 2) + n, -7, dtype=torch.int32, device=DEV)
        cf.cf_sample_lp(emb, seed, 0, R, cf.CF_F32, fields, cf.make_lp(sigma2, nbar, c, pseed), ws, wsb)
        torch.cuda.synchronize()
        counts[name] = c
    assert all(int(c.min()) >= 0 for c in counts.values())
    if len(counts) == 2:
        assert torch.equal(counts["list"], counts["in_place"])
    fl, nd = _lp_check(orc, fields.double().cpu().numpy().reshape(2 * R, -1),
                       counts["list"].cpu().numpy().reshape(2 * R, -1), None, sigma2, nbar, None, pseed, 0)
    print("flagged %d, differing %d" % (fl, nd))
    emb.close()


PK_CASES = [((64, 64), 16, cf.CF_BINS_LINEAR), ((32, 32), 5, cf.CF_BINS_LOG), ((16, 16, 16), 8, cf.CF_BINS_LINEAR),
            ((128, 128), 64, cf.CF_BINS_LINEAR), ((8, 8), 3, cf.CF_BINS_LINEAR)]


@pytest.mark.parametrize("n,nbins,kind", PK_CASES)
@pytest.mark.parametrize("dt", [cf.CF_F32, cf.CF_F64])
def test_power_spectrum_parity(orc, n, nbins, kind, dt):
    F = 7  # odd: the last field is transformed with a zero partner
    x = W.gaussian_field_values((F,) + n, seed=41, scale=1.3)
    tdt = torch.float32 if dt == cf.CF_F32 else torch.float64
    xt = torch.from_numpy(x).to(tdt).to(DEV)
    cell = 0.5
    g = cf.make_grid(n, [cell] * len(n))
    kmin = 1.0 if kind == cf.CF_BINS_LOG else 0.0
    bins = cf.make_bins(nbins, kind, kmin, 0.0)
    wsb = cf.cf_power_spectrum_workspace_size(g, F, bins, dt)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    pk = torch.empty((F, nbins), dtype=torch.float64, device=DEV)
    nm = torch.empty(nbins, dtype=torch.int64, device=DEV)
    mean = torch.empty(nbins, dtype=torch.float64, device=DEV)
    cov = torch.empty((nbins, nbins), dtype=torch.float64, device=DEV)
    cf.cf_power_spectrum(xt, dt, g, F, bins, pk, nm, mean, cov, ws, wsb)
    torch.cuda.synchronize()
    edges = orc.bin_edges(orc.BINS_LOG if kind == cf.CF_BINS_LOG else orc.BINS_LINEAR, nbins, kmin, n[0] / 2)
    opk, onm = orc.power_spectrum(xt.double().cpu().numpy(), n, edges, cell=cell)
    assert np.array_equal(nm.cpu().numpy(), onm)
    tol = 2e-5 if dt == cf.CF_F32 else 1e-10
    assert np.allclose(pk.cpu().numpy(), opk, rtol=tol, atol=tol * opk.max() * 1e-3)
    om, oc = orc.mean_cov(opk)
    assert np.allclose(mean.cpu().numpy(), om, rtol=tol, atol=1e-300)
    assert np.allclose(cov.cpu().numpy(), oc, rtol=10 * tol, atol=10 * tol * np.abs(oc).max())


@pytest.mark.parametrize("n,F,masked", [((64, 64), 6, True), ((64, 64), 6, False), ((16, 16, 16), 5, True),
                                         ((32, 32), 5, False)])
def test_power_spectrum_counts_parity(orc, n, F, masked):
    f = W.survey_mask(n, seed=51) if masked else np.ones(n, dtype=np.float32)
    counts = np.random.default_rng(52).poisson(3.0 * f, size=(F,) + n).astype(np.int32)
    g = cf.make_grid(n)
    nb = 16 if len(n) == 2 else 8
    bins = cf.make_bins(nb)
    wsb = cf.cf_power_spectrum_workspace_size(g, F, bins, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    pk = torch.empty((F, nb), dtype=torch.float64, device=DEV)
    nm = torch.empty(nb, dtype=torch.int64, device=DEV)
    mean = torch.empty(nb, dtype=torch.float64, device=DEV)
    ct = torch.from_numpy(counts).to(DEV)
    ft = torch.from_numpy(f).to(DEV) if masked else None
    cf.cf_power_spectrum_counts(ct, ft, g, F, bins, pk, nm, mean, None, ws, wsb)
    torch.cuda.synchronize()
    dg = orc.counts_to_delta(counts.reshape(F, -1), f.ravel().astype(np.float64) if masked else None)
    opk, onm = orc.power_spectrum(dg.reshape((F,) + n), n, orc.bin_edges(0, nb, 0.0, n[0] / 2))
    assert np.array_equal(nm.cpu().numpy(), onm)
    assert np.allclose(pk.cpu().numpy(), opk, rtol=2e-5, atol=1e-7 * opk.max())
    assert np.allclose(mean.cpu().numpy(), opk.mean(0), rtol=2e-5)


@pytest.mark.parametrize("box_factor,log1p", [(1, False), (2, True), (4, False)])
def test_periodic_box_embedding(orc, box_factor, log1p):
    """cf_embed_periodic: the box eigenvalues equal the oracle's (section 3.3)."""
    n = (32, 64)
    flags = cf.CF_EMBED_CLAMP | (cf.CF_EMBED_LOG1P if log1p else 0)
    emb = cf.cf_embed_periodic(cf.make_grid(n), cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.5, 4.0, 0.4), box_factor, 2, 4,
                               flags)
    ref = orc.periodic_lambda(n, cf.CF_XI_GEN_CAUCHY, 0.5, 4.0, 0.4, box_factor, 2, 4, log1p=log1p)
    lam = torch.empty(ref.shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    assert np.max(np.abs(lam.cpu().numpy() - ref)) <= 1e-12 * np.abs(ref).max()
    # the sampler runs on it: fields of n (2n for box_factor 4) per axis
    R = 2
    out_n = tuple(2 * v for v in n) if box_factor == 4 else n
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + out_n, dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, 3, 0, R, cf.CF_F32, fields, ws, wsb)
    torch.cuda.synchronize()
    assert torch.isfinite(fields).all()
    if box_factor == 4:  # the survey corner of the 2n field
        corner = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
        cf.cf_copy_corner(fields, cf.CF_F32, cf.make_grid(out_n), cf.make_grid(n), 2 * R, corner)
        torch.cuda.synchronize()
        assert torch.equal(corner, fields[:, :, : n[0], : n[1]])
    emb.close()


def test_workspace_of_the_reported_size_takes_one_chunk():
    """A workspace of cf_sample_workspace_size(R) bytes holds all R
    realizations of a small grid at once (with the list of deferred Poisson
    decisions): one launch of each pass, no ragged tail chunk."""
    n, R = (128, 128), 64
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 0.8, 3.0))
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    cf.cf_kernel_timing(1)
    cf.cf_sample_lp(emb, 3, 0, R, cf.CF_F32, fields, cf.make_lp(0.8, 2.0, counts, 4), ws, wsb)
    torch.cuda.synchronize()
    t = cf.cf_kernel_timing_read()
    cf.cf_kernel_timing(0)
    launches = {k.split("<")[0]: v[0] for k, v in t.items()}
    assert launches.get("sample_rows_f32") == 1 and launches.get("icols_fields_lp_f32") == 1, launches
    assert launches.get("poisson_fixup") == 1, launches
    emb.close()


@pytest.mark.parametrize("n,kind,amp,scale,beta,clamp", [((512, 512), 1, 0.8, 8.0, 0.4, True),
                                                         ((64, 64), 0, 1.0, 4.0, 0.0, False),
                                                         ((128, 128, 128), 2, 1.0, 6.0, 0.0, False),
                                                         ((16, 32), 2, 1.3, 1.5, 0.0, False)])
def test_double_float_embedding(orc, n, kind, amp, scale, beta, clamp):
    """CF_EMBED_DF: eigenvalues through double-float transforms within the
    1e-12 lambda_max gate of the oracle's binary64 ones, the same threshold
    decisions, and binary32 fields within the binary32 gate end to end."""
    o = orc.embed(list(n), kind, amp, scale, beta, clamp=clamp)
    flags = cf.CF_EMBED_DF | (cf.CF_EMBED_CLAMP if clamp else 0)
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(kind, amp, scale, beta), flags)
    lam = torch.empty(o["lambda"].shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    lmax = o["lambda"].max()
    err = float(np.max(np.abs(lam.cpu().numpy() - o["lambda"])) / lmax)
    print("double-float eigenvalues: max error %.2e lambda_max" % err)
    assert err <= 1e-12
    assert emb.report["n_negative"] == o["report"]["n_negative"]
    if o["report"]["clamped"]:
        assert emb.report["cov_error"] == pytest.approx(o["report"]["cov_error"], rel=1e-6, abs=1e-13)
    R = 2
    got = _fields(emb, 91, 4, R, cf.CF_F32, n).double().cpu().numpy()
    ref = orc.sample(n, o["sqrt_lambda"], 91, 4, R, 1)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    emb.close()
