"""GPU parity of the binary32 row pass for rows of 1024 points (one warp per
row) and of 256 points (two rows per warp), section 2, eq. (Papos2): noise,
sqrt(lambda+) scaling and the inverse transform of the last axis, keeping
the survey's half.  Fields against the oracle's sampler at the binary32 gate
(relative L2 1e-5) for 2D surveys, 3D grids whose last axis has 1024 or 256
points, and a survey embedded in four times its side (256 of 1024 outputs
kept); every CTA shape gives the same bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _sample(emb, n, seed, r0, R):
    wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + tuple(n), dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, seed, r0, R, cf.CF_F32, out, ws, wsb)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,factor,kind,amp,scale,beta,seed,r0,R", [
    ((512, 512), 2, cf.CF_XI_GEN_CAUCHY, 0.8, 8.0, 0.4, 2, 0, 3),
    ((3, 5, 512), 2, cf.CF_XI_EXPONENTIAL, 1.0, 3.0, 0.0, 0xFEEDFACE12, 2**32 - 3, 3),
    ((256, 256), 4, cf.CF_XI_GAUSSIAN, 1.0, 6.0, 0.0, 9, 41, 2),
    ((128, 128), 2, cf.CF_XI_GEN_CAUCHY, 1.2, 4.0, 0.4, 12, 7, 3),
    ((32, 32, 128), 2, cf.CF_XI_EXPONENTIAL, 1.0, 6.0, 0.0, 3, 0, 2),
])
def test_warp_row_pass_matches_the_oracle(orc, n, factor, kind, amp, scale, beta, seed, r0, R):
    emb = cf.cf_embed(cf.make_grid(n, factor=factor), cf.make_xi(kind, amp, scale, beta), cf.CF_EMBED_CLAMP)
    got = _sample(emb, n, seed, r0, R).double().cpu().numpy()
    M = [int(2 ** np.ceil(np.log2(factor * v))) for v in n]  # sides embedded in powers of two
    assert M[-1] in (256, 1024)
    o = orc.embed(list(n), kind, amp, scale, beta, clamp=True, M=M)
    ref = orc.sample(n, o["sqrt_lambda"], seed, r0, R, 1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    # every realization and both fields of each, not just the total
    for r in range(R):
        for h in range(2):
            e = np.linalg.norm(got[r, h] - ref[r, h]) / np.linalg.norm(ref[r, h])
            assert e <= 1e-5, (r, h, e)
    emb.close()


@pytest.mark.parametrize("n", [(1, 512), (3, 10, 512), (1, 128), (3, 10, 128)])
def test_warp_row_pass_cta_shapes_give_the_same_bits(n):
    """8, 4 or 16 warps per CTA: 2 rows (fewer than the warps of any shape)
    and 256 rows, of 1024 and of 256 points, two chunkings, identical
    fields."""
    R = 5
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_EXPONENTIAL, 1.0, 3.0), cf.CF_EMBED_CLAMP)
    ref = _sample(emb, n, 5, 7, R)
    for rs in range(3):
        for chunk in (0, 2):
            cf.cf_tune_set(emb, cf.CF_F32, chunk, rs, 0)
            assert torch.equal(_sample(emb, n, 5, 7, R), ref), (rs, chunk)
    cf.cf_tune_set(emb, cf.CF_F32, 0, 0, 0)
    emb.close()
