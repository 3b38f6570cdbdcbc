"""GPU tests of the sampler's autotuner: it picks one of the candidate chunks
and CTA shapes, the chosen schedule is used afterwards (the workspace size
follows it), and no schedule changes a result bit (chunking and the CTA
shape of the paired passes leave every operation of every output as it
is)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _run(emb, n, R, dt, ws_bytes):
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + n, dtype=torch.float32 if dt == cf.CF_F32 else torch.float64, device=DEV)
    cf.cf_sample(emb, 77, 3, R, dt, out, ws, ws_bytes)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,dt", [((64, 128), cf.CF_F32), ((16, 8, 32), cf.CF_F64)])
def test_tuned_chunk_is_used_and_changes_no_result(n, dt):
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 3.0), cf.CF_EMBED_CLAMP)
    R = 9
    before = _run(emb, n, R, dt, cf.cf_sample_workspace_size(emb, R, dt))
    per = cf.cf_sample_workspace_size(emb, 1, dt)
    ws_cap = per * 8  # candidates 1, 2, 4, 8
    ws = torch.empty(ws_cap, dtype=torch.uint8, device=DEV)
    scratch = torch.empty((R, 2) + n, dtype=before.dtype, device=DEV)
    chunk, ms = cf.cf_tune_sample(emb, dt, R, ws, ws_cap, scratch)
    assert chunk in (1, 2, 4, 8) and ms > 0
    # the workspace for R realizations is now the one of a tuned chunk
    assert cf.cf_sample_workspace_size(emb, R, dt) == cf.cf_sample_workspace_size(emb, chunk, dt)
    assert cf.cf_sample_workspace_size(emb, R, dt) <= per * chunk
    after = _run(emb, n, R, dt, cf.cf_sample_workspace_size(emb, R, dt))
    assert torch.equal(before, after)
    emb.close()


def test_tune_rejects_bad_arguments():
    emb = cf.cf_embed(cf.make_grid((32, 32)), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    with pytest.raises(cf.CfError) as ei:
        cf.cf_tune_sample(emb, cf.CF_F32, 0, None, 0, None)
    assert ei.value.status == cf.CF_ERR_ARG
    emb.close()


def _run_lp(emb, n, R, ws_bytes):
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    counts = torch.empty((R, 2) + n, dtype=torch.int32, device=DEV)
    cf.cf_sample_lp(emb, 91, 5, R, cf.CF_F32, out, cf.make_lp(0.8, 2.0, counts, 92), ws, ws_bytes)
    torch.cuda.synchronize()
    return out, counts


@pytest.mark.parametrize("n,R", [((256, 256), 5), ((128, 64, 128), 3)])
def test_every_cta_shape_gives_the_same_bits(n, R):
    """The paired binary32 passes compute every output with the same
    operations whatever the CTA shape: all 3 x 3 row/column shapes (and a
    chunk of two realizations, with its odd tail) give identical fields and
    counts."""
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 3.0), cf.CF_EMBED_CLAMP)
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ref_f, ref_c = _run_lp(emb, n, R, wsb)
    for rs in range(3):
        for cs in range(3):
            for chunk in (0, 2):
                cf.cf_tune_set(emb, cf.CF_F32, chunk, rs, cs)
                assert cf.cf_tune_info(emb, cf.CF_F32) == (chunk, rs, cs, 0)
                f, c = _run_lp(emb, n, R, cf.cf_sample_workspace_size(emb, R, cf.CF_F32))
                assert torch.equal(f, ref_f), (rs, cs, chunk)
                assert torch.equal(c, ref_c), (rs, cs, chunk)
    cf.cf_tune_set(emb, cf.CF_F32, 0, 0, 0)
    assert cf.cf_tune_info(emb, cf.CF_F32) == (0, 0, 0, 0)
    emb.close()


def test_tuner_picks_shapes_and_changes_no_result():
    n, R = (256, 256), 8
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 4.0))
    before = _run(emb, n, R, cf.CF_F32, cf.cf_sample_workspace_size(emb, R, cf.CF_F32))
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(wsb, dtype=torch.uint8, device=DEV)
    scratch = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    chunk, ms = cf.cf_tune_sample(emb, cf.CF_F32, R, ws, wsb, scratch)
    c, rs, cs, _ = cf.cf_tune_info(emb, cf.CF_F32)
    assert c == chunk and 0 <= rs < 3 and 0 <= cs < 3 and ms > 0
    after = _run(emb, n, R, cf.CF_F32, cf.cf_sample_workspace_size(emb, R, cf.CF_F32))
    assert torch.equal(before, after)
    cf.cf_tune_set(emb, cf.CF_F32)
    emb.close()


def test_tune_set_rejects_bad_shapes():
    emb = cf.cf_embed(cf.make_grid((32, 32)), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    for args in ((0, 3, 0), (0, 0, -1), (-1, 0, 0), (0, 0, 0, 2)):
        with pytest.raises(cf.CfError) as ei:
            cf.cf_tune_set(emb, cf.CF_F32, *args)
        assert ei.value.status == cf.CF_ERR_ARG
    big = cf.cf_embed(cf.make_grid((256, 256)), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 2.0))
    with pytest.raises(cf.CfError) as ei:  # no persistent sampler for 512^2 embeddings
        cf.cf_tune_set(big, cf.CF_F32, 0, 0, 0, 1)
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    emb.close()
    big.close()


@pytest.mark.parametrize("n,R,lp", [((64, 64), 5, True), ((32, 64), 3, False), ((32, 32, 32), 4, True),
                                    ((64, 64, 64), 3, True), ((20, 50), 2, True)])
def test_persistent_sampler_gives_the_same_bits(n, R, lp):
    """The whole chunk in one cooperative launch (rows, a grid-wide barrier,
    the column passes, the deferred binary64 decisions) runs the same tiles
    as the separate launches: identical fields and counts, for whole and
    chunked batches (an odd tail included)."""
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.9, 3.0, 0.4), cf.CF_EMBED_CLAMP)
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ref = _run_lp(emb, n, R, wsb) if lp else (_run(emb, n, R, cf.CF_F32, wsb), None)
    for chunk in (0, 2):
        cf.cf_tune_set(emb, cf.CF_F32, chunk, 0, 0, 1)
        assert cf.cf_tune_info(emb, cf.CF_F32)[3] == 1
        wsb2 = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
        got = _run_lp(emb, n, R, wsb2) if lp else (_run(emb, n, R, cf.CF_F32, wsb2), None)
        assert torch.equal(got[0], ref[0]), chunk
        if lp:
            assert torch.equal(got[1], ref[1]), chunk
    cf.cf_tune_set(emb, cf.CF_F32)
    emb.close()
