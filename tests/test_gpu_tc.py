"""GPU tests of the tensor-core sampler modes (CF_BF16_TC, CF_F16_TC).

These modes round the data to 16 bits before every DFT-matrix stage, so they
are not bit-for-bit comparable with the oracle: the error against the oracle's
binary64 fields (same binary32 noise) is bounded by the rounding analysis
instead.  With unit roundoff u (bf16 2^-8, fp16 2^-11) and dS roundings of
the data (S radix-16 stages per axis, d axes), each contributing at most u
relative (about u/sqrt(3) RMS), the relative L2 error stays below u*sqrt(dS).  The
error must also exceed u/64: a smaller one would mean the 16-bit stages did
not run.  Every run also checks that no tensor-core wait ran out of time.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")
U = {cf.CF_BF16_TC: 2.0 ** -8, cf.CF_F16_TC: 2.0 ** -11}


def _tc_fields(emb, seed, r0, R, dt, n, ws_bytes=None):
    need = cf.cf_sample_workspace_size(emb, R, dt)
    ws_bytes = need if ws_bytes is None else ws_bytes
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=DEV)
    out = torch.empty((R, 2) + tuple(n), dtype=torch.float32, device=DEV)
    cf.cf_sample(emb, seed, r0, R, dt, out, ws, ws_bytes)
    assert cf.cf_tc_faults() == 0
    return out


def _roundings(n):
    # rounding stages per axis: 2 radix-16 stages for 256 points, 3 for 4096,
    # and a binary32 first radix (2, 4 or 8) before 2 radix-16 stages
    # otherwise; every axis counts with the largest
    return len(n) * max(2 if 2 * v == 256 else 3 for v in n)


CASES = [((128, 128), cf.CF_XI_GAUSSIAN, 4.0, 0.0, False),
         ((128, 2048), cf.CF_XI_EXPONENTIAL, 6.0, 0.0, False),
         ((2048, 128), cf.CF_XI_GEN_CAUCHY, 8.0, 0.4, True),
         ((256, 512), cf.CF_XI_GEN_CAUCHY, 8.0, 0.4, True),    # first radix 2 and 4
         ((1024, 128), cf.CF_XI_EXPONENTIAL, 5.0, 0.0, False),  # first radix 8
         ((512, 512), cf.CF_XI_GEN_CAUCHY, 8.0, 0.4, True),     # the 2D 512^2 workload's grid
         ((128, 128, 128), cf.CF_XI_EXPONENTIAL, 4.0, 0.0, True),  # 3D: three passes
         ((256, 128, 128), cf.CF_XI_GEN_CAUCHY, 6.0, 0.4, True),   # 3D, first radix 2 on axis 0
         ((128, 128, 512), cf.CF_XI_GAUSSIAN, 5.0, 0.0, True)]     # 3D, first radix 4 on the rows


@pytest.mark.parametrize("dt", [cf.CF_BF16_TC, cf.CF_F16_TC])
@pytest.mark.parametrize("n,kind,scale,beta,clamp", CASES)
def test_tc_fields_within_rounding_bound(orc, n, kind, scale, beta, clamp, dt):
    o = orc.embed(list(n), kind, 0.8, scale, beta, clamp=clamp)
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(kind, 0.8, scale, beta), cf.CF_EMBED_CLAMP if clamp else 0)
    seed, r0, R = 0xABCDEF12345, 7, 3
    got = _tc_fields(emb, seed, r0, R, dt, n).double().cpu().numpy()
    ref = orc.sample(n, o["sqrt_lambda"], seed, r0, R, 1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    u = U[dt]
    assert u / 64 < err <= u * np.sqrt(_roundings(n)), err
    # each realization separately (no cross-talk between lines, blocks or chunks)
    for r in range(R):
        e = np.linalg.norm(got[r] - ref[r]) / np.linalg.norm(ref[r])
        assert e <= u * np.sqrt(_roundings(n)), (r, e)
    emb.close()


def test_precision_sweep_errors(orc):
    """2D 2048^2 survey in 4096^2 (the precision-sweep workload), realization 5
    of seed 4 in every precision: relative L2 error of the fields and largest
    relative error of the binned power spectrum against the oracle in binary64
    on the same noise (binary64 noise for CF_F64, binary32 noise otherwise).
    Prints one JSON line with the table."""
    import json
    n = (2048, 2048)
    nbins = 64
    o = orc.embed(list(n), cf.CF_XI_GEN_CAUCHY, 0.8, 16.0, 0.4, clamp=True)
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GEN_CAUCHY, 0.8, 16.0, 0.4), cf.CF_EMBED_CLAMP)
    edges = orc.bin_edges(orc.BINS_LINEAR, nbins, 0.0, n[0] / 2)
    refs = {}
    table = {}
    bound = {cf.CF_F64: 1e-10, cf.CF_F32: 1e-5, cf.CF_BF16_TC: U[cf.CF_BF16_TC] * np.sqrt(6),
             cf.CF_F16_TC: U[cf.CF_F16_TC] * np.sqrt(6)}
    for name, dt in (("f64", cf.CF_F64), ("f32", cf.CF_F32), ("bf16_tc", cf.CF_BF16_TC), ("f16_tc", cf.CF_F16_TC)):
        noise = 0 if dt == cf.CF_F64 else 1
        if noise not in refs:
            ref = orc.sample(n, o["sqrt_lambda"], 4, 5, 1, noise)[0]
            refs[noise] = (ref, orc.power_spectrum(ref, n, edges)[0])
        ref, ref_pk = refs[noise]
        if dt in (cf.CF_BF16_TC, cf.CF_F16_TC):
            got = _tc_fields(emb, 4, 5, 1, dt, n)[0]
        else:
            wsb = cf.cf_sample_workspace_size(emb, 1, dt)
            ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
            got = torch.empty((1, 2) + n, dtype=torch.float64 if dt == cf.CF_F64 else torch.float32, device=DEV)
            cf.cf_sample(emb, 4, 5, 1, dt, got, ws, wsb)
            got = got[0]
        g = got.double().cpu().numpy()
        err = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
        pk = orc.power_spectrum(g, n, edges)[0]
        pk_err = float(np.max(np.abs(pk - ref_pk) / np.abs(ref_pk)))
        table[name] = {"field_rel_l2": err, "pk_max_rel": pk_err}
        assert err <= bound[dt], (name, err)
        if dt in (cf.CF_BF16_TC, cf.CF_F16_TC):
            assert U[dt] / 64 < err, (name, err)
    print("\nPRECISION_SWEEP " + json.dumps(table))
    emb.close()


@pytest.mark.parametrize("n", [(128, 128), (128, 128, 128)])
def test_tc_deterministic_and_chunk_independent(n):
    emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
    for dt in (cf.CF_BF16_TC, cf.CF_F16_TC):
        a = _tc_fields(emb, 9, 10, 5, dt, n)
        b = _tc_fields(emb, 9, 10, 5, dt, n)
        assert torch.equal(a, b)
        one = cf.cf_sample_workspace_size(emb, 1, dt)
        c = _tc_fields(emb, 9, 10, 5, dt, n, ws_bytes=2 * one)  # chunks of 2, ragged last
        assert torch.equal(a, c)
        d = _tc_fields(emb, 9, 13, 1, dt, n)  # realization 13 alone
        assert torch.equal(a[3:4], d)
    emb.close()


def test_tc_unsupported_and_errors():
    for n in ((64, 64), (128, 64, 128), (256,)):  # sides 128: too short; 1D
        emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
        with pytest.raises(cf.CfError) as ei:
            cf.cf_sample_workspace_size(emb, 1, cf.CF_BF16_TC)
        assert ei.value.status == cf.CF_ERR_UNSUPPORTED
        emb.close()
    emb = cf.cf_embed(cf.make_grid((128, 128)), cf.make_xi(cf.CF_XI_GAUSSIAN, 1.0, 3.0))
    out = torch.empty((1, 2, 128, 128), dtype=torch.float32, device=DEV)
    ws = torch.empty(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.cf_sample(emb, 1, 0, 1, cf.CF_F16_TC, out, ws, 64)
    assert ei.value.status == cf.CF_ERR_NOMEM
    counts = torch.empty((1, 2, 128, 128), dtype=torch.int32, device=DEV)
    with pytest.raises(cf.CfError) as ei:
        cf.cf_sample_lp(emb, 1, 0, 1, cf.CF_BF16_TC, out, cf.make_lp(0.5, 1.0, counts, 3), ws, 64)
    assert ei.value.status == cf.CF_ERR_UNSUPPORTED
    emb.close()
