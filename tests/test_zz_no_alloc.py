"""cf_sample_noalloc: the binary32 sampler for callers that cannot allocate
device memory where they sample (for example while another thread captures a
CUDA graph in global mode, or under a fixed device-memory budget).  It must
give the same fields as cf_sample with a caller workspace, on two calls in a
row (the second call finds the previous call's data in the shared static
array), and reject grids whose realization does not fit the array.

This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _rel_l2(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _reference(emb, seed, r0, R, n):
    ws_bytes = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, seed, r0, R, cf.CF_F32, out, ws, ws_bytes)
    return out


@pytest.mark.parametrize("n", [(64, 64), (256, 128), (16, 16, 32)])
def test_noalloc_matches_workspace_sampler_twice(n):
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 2.0))
    for seed, r0, R in ((7, 0, 3), (8, 40, 5)):
        ref = _reference(emb, seed, r0, R, n)
        got = torch.full_like(ref, float("nan"))
        cf.cf_sample_noalloc(emb, seed, r0, R, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel_l2(got, ref) <= 1e-5
    emb.close()


def test_noalloc_takes_no_device_memory():
    """After the first call (its one-time set-up), further calls leave the
    device's free memory as it is: nothing is allocated or freed."""
    n, R = (128, 64), 4
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
    out = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
    cf.cf_sample_noalloc(emb, 5, 0, R, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(DEV)
    for k in range(3):
        cf.cf_sample_noalloc(emb, 6 + k, 10 * k, R, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0
    emb.close()


def test_noalloc_rejects_grids_beyond_the_static_array():
    # 3D 64x64x128: one realization needs 24 MiB of intermediate
    emb = cf.cf_embed(cf.make_grid((64, 64, 128)), cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 2.0))
    out = torch.empty(8, dtype=torch.float32, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.cf_sample_noalloc(emb, 1, 0, 1, out)
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    assert "static scratch" in str(ei.value)
    emb.close()
