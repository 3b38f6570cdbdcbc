"""GPU parity of embeddings on grids larger than twice the survey side
(cf_grid.embed_factor 4 and 8) and of survey sizes that are not powers of two
(embedded in the next power of two): eigenvalues, report and fields against
the oracle with the same embedded grid, counts of the fused lognormal +
Poisson step, captured plans and the serving loop on such grids, and the
calls that refuse them.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _m(n, p):
    """Embedded sides: the smallest power of two >= p n per axis."""
    return tuple(1 << int(np.ceil(np.log2(p * v))) for v in n)


CASES = [((64,), 8, cf.CF_XI_GAUSSIAN, 3.0, 0.0, False),
         ((100,), 2, cf.CF_XI_GAUSSIAN, 4.0, 0.0, False),         # survey sizes that are not powers of two
         ((48, 80), 2, cf.CF_XI_EXPONENTIAL, 3.0, 0.0, False),
         ((100, 100), 4, cf.CF_XI_GEN_CAUCHY, 6.0, 0.4, True),
         ((24, 40, 12), 2, cf.CF_XI_EXPONENTIAL, 2.0, 0.0, False),
         ((5, 3), 8, cf.CF_XI_GAUSSIAN, 0.8, 0.0, False),
         ((32, 64), 4, cf.CF_XI_EXPONENTIAL, 2.0, 0.0, False),
         ((16, 16), 8, cf.CF_XI_GEN_CAUCHY, 2.0, 0.4, True),    # not PSD at any factor: clamped
         ((64, 64), 4, cf.CF_XI_GEN_CAUCHY, 8.0, 0.4, True),
         ((8, 16, 8), 4, cf.CF_XI_EXPONENTIAL, 1.0, 0.0, False),
         ((2, 4), 8, cf.CF_XI_GAUSSIAN, 0.6, 0.0, False)]


@pytest.mark.parametrize("n,p,kind,scale,beta,clamp", CASES)
def test_padded_embedding_and_fields(orc, n, p, kind, scale, beta, clamp):
    o = orc.embed(list(n), kind, 0.9, scale, beta, clamp=clamp, M=_m(n, p))
    g = cf.make_grid(n, factor=p)
    emb = cf.cf_embed(g, cf.make_xi(kind, 0.9, scale, beta), cf.CF_EMBED_CLAMP if clamp else 0)
    lam = torch.empty(o["lambda"].shape, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    lmax = o["lambda"].max()
    assert np.max(np.abs(lam.cpu().numpy() - o["lambda"])) <= 1e-12 * lmax
    assert emb.report["n_negative"] == o["report"]["n_negative"]
    if o["report"]["clamped"]:
        assert emb.report["cov_error"] == pytest.approx(o["report"]["cov_error"], rel=1e-6, abs=1e-13)
    # fields, fed the oracle's eigenvalues (identical threshold decisions)
    emb2 = cf.cf_embed_from_lambda(g, torch.from_numpy(o["lambda"]).to(DEV), cf.CF_EMBED_CLAMP)
    seed, r0, R = 0xC0FFEE + p, 3, 3
    for dt, odt, tol in ((cf.CF_F64, 0, 1e-10), (cf.CF_F32, 1, 1e-5)):
        wsb = cf.cf_sample_workspace_size(emb2, R, dt)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
        out = torch.empty((R, 2) + tuple(n), dtype=torch.float32 if dt == cf.CF_F32 else torch.float64, device=DEV)
        cf.cf_sample(emb2, seed, r0, R, dt, out, ws, wsb)
        torch.cuda.synchronize()
        ref = orc.sample(n, o["sqrt_lambda"], seed, r0, R, odt)
        assert rel_l2(out.double().cpu().numpy(), ref) <= tol, (dt, rel_l2(out.double().cpu().numpy(), ref))
    emb.close()
    emb2.close()


@pytest.mark.parametrize("n,p", [((32, 32), 4), ((100, 60), 2)])
def test_padded_fused_counts_plan_and_serving(orc, n, p):
    R = 3
    g = cf.make_grid(n, factor=p)
    emb = cf.cf_embed(g, cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 4.0, 0.4), cf.CF_EMBED_CLAMP)
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    plain = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, 41, 6, R, cf.CF_F32, plain, ws, wsb)
    fields = torch.empty_like(plain)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    cf.cf_sample_lp(emb, 41, 6, R, cf.CF_F32, fields, cf.make_lp(0.8, 3.0, counts, 42), ws, wsb)
    torch.cuda.synchronize()
    assert torch.equal(fields, plain)
    Gd = fields.double().cpu().numpy().reshape(2 * R, -1)
    _, oc, margin = orc.lognormal_poisson(Gd, 0.8, 3.0, seed=42, field0=12)
    c = counts.cpu().numpy().reshape(oc.shape)
    assert not ((c != oc) & (margin >= 1e-6)).any()
    # a captured plan draws the same realizations
    pf = torch.empty_like(plain)
    plan = cf.Plan(emb, 41, 6, R, pf)
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(pf, plain)
    plan.close()
    # the serving loop on the same grid and spectrum (amplitude applied at
    # sampling: equal to rounding)
    sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=1))
    host = torch.empty((R, 2) + n, dtype=torch.float32).pin_memory()
    t = cf.cf_serve_submit(sv, cf.make_request(n, cf.CF_XI_GEN_CAUCHY, 0.8, 4.0, 0.4, seed=41, r0=6, R=R,
                                               host_fields=host, factor=p))
    res = cf.cf_serve_wait(sv, t, 30_000_000)
    assert res["status"] == cf.CF_OK
    got, ref = host.double().numpy(), plain.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    cf.cf_serve_release(sv, t)
    cf.cf_serve_destroy(sv)
    emb.close()


def test_padded_grid_refusals():
    with pytest.raises(cf.CfError) as ei:
        cf.cf_embed(cf.make_grid((32, 32), factor=3), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    assert ei.value.status == cf.CF_ERR_ARG
    with pytest.raises(cf.CfError) as ei:  # 8 * 1024 exceeds the longest line
        cf.cf_embed(cf.make_grid((1024,), factor=8), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    for n, p in (((128, 128), 4), ((200, 256), 2)):  # tensor-core modes need M = 2n
        emb = cf.cf_embed(cf.make_grid(n, factor=p), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
        with pytest.raises(cf.CfError) as ei:
            cf.cf_sample_workspace_size(emb, 1, cf.CF_BF16_TC)
        assert ei.value.status == cf.CF_ERR_UNSUPPORTED
        emb.close()
    for n, p in (((32, 32), 4), ((30, 32), 2)):
        with pytest.raises(cf.CfError) as ei:
            cf.cf_embed_periodic(cf.make_grid(n, factor=p), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0), 2, 4, 2)
        assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    # the power spectrum takes any side up to 2048 (Bluestein) or 4096 (powers of two)
    bins = cf.make_bins(4)
    assert cf.cf_power_spectrum_workspace_size(cf.make_grid((100, 100)), 2, bins, cf.CF_F32) > 0
    with pytest.raises(cf.CfError) as ei:
        cf.cf_power_spectrum_workspace_size(cf.make_grid((3000, 100)), 2, bins, cf.CF_F32)
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED


def test_padded_masked_counts_and_double_float(orc):
    """A padded, non-power-of-two grid with a survey mask in the fused
    lognormal + Poisson step, and the double-float eigenvalue transforms on a
    padded grid."""
    from paper_1406_6072_gb300 import workloads as W
    n, p, R = (48, 80), 4, 2
    g = cf.make_grid(n, factor=p)
    M = _m(n, p)
    o = orc.embed(list(n), cf.CF_XI_GEN_CAUCHY, 0.8, 4.0, 0.4, clamp=True, M=M)
    emb = cf.cf_embed(g, cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 4.0, 0.4), cf.CF_EMBED_CLAMP | cf.CF_EMBED_DF)
    lam = torch.empty(M, dtype=torch.float64, device=DEV)
    cf.cf_embedding_lambda(emb, lam)
    torch.cuda.synchronize()
    assert np.max(np.abs(lam.cpu().numpy() - o["lambda"])) <= 1e-12 * o["lambda"].max()
    f = W.survey_mask(n, seed=17)
    ft = torch.from_numpy(f).to(DEV)
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    fields = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    cf.cf_sample_lp(emb, 5, 0, R, cf.CF_F32, fields, cf.make_lp(0.8, 3.0, counts, 6, f=ft), ws, wsb)
    torch.cuda.synchronize()
    ref = orc.sample(n, o["sqrt_lambda"], 5, 0, R, 1)
    assert rel_l2(fields.double().cpu().numpy(), ref) <= 1e-5
    Gd = fields.double().cpu().numpy().reshape(2 * R, -1)
    _, oc, margin = orc.lognormal_poisson(Gd, 0.8, 3.0, f=f.ravel().astype(np.float64), seed=6, field0=0)
    c = counts.cpu().numpy().reshape(oc.shape)
    assert not ((c != oc) & (margin >= 1e-6)).any()
    emb.close()
