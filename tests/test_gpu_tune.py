"""GPU tests of the sampler's chunk autotuner: it picks one of the candidate
chunks, the chosen schedule is used afterwards (the workspace size follows
it), and tuning changes no result (chunking never changes a field bit)."""
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
