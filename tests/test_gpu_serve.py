"""GPU tests of the serving loop: served results equal cf_sample's (the
embedding is cached at amplitude 1 and scaled by sqrt(amp), so within the
binary32 field tolerance), a request gives the same result alone and in a
mixed, batched stream (bit for bit), served counts match the stand-alone
lognormal/Poisson step, failures come back as statuses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402

DEV = torch.device("cuda:0")


def _host(shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype).pin_memory()


REQS = [((64, 64), cf.CF_XI_GAUSSIAN, 0.7, 3.0, 0.0, 11, 0, 3),
        ((64, 64), cf.CF_XI_GEN_CAUCHY, 1.3, 4.0, 0.4, 12, 5, 2),
        ((32, 32, 32), cf.CF_XI_EXPONENTIAL, 0.5, 2.0, 0.0, 13, 2, 2),
        ((128, 128), cf.CF_XI_GAUSSIAN, 1.1, 3.0, 0.0, 14, 7, 4),
        ((64, 64), cf.CF_XI_GAUSSIAN, 0.2, 3.0, 0.0, 15, 100, 1),
        ((256,), cf.CF_XI_EXPONENTIAL, 1.5, 6.0, 0.0, 16, 3, 5)]


def _serve(sv, specs, want_counts=False, first=None):
    """Serves specs (host buffers pinned up front); `first` is submitted just
    before them.  Returns (results, host outputs, ticket of `first`)."""
    tickets, outs, reqs = [], [], []
    for n, kind, amp, scale, beta, seed, r0, R in specs:
        hf = _host((R, 2) + n)
        hc = _host((R, 2) + n, torch.int32) if want_counts else None
        reqs.append(cf.make_request(n, kind, amp, scale, beta, seed=seed, r0=r0, R=R, want_counts=want_counts,
                                    sigma2=amp, nbar=2.0, lp_seed=seed + 1, host_fields=hf, host_counts=hc))
        outs.append((hf, hc))
    t_first = cf.cf_serve_submit(sv, first) if first is not None else None
    for req in reqs:
        tickets.append(cf.cf_serve_submit(sv, req))
    res = [cf.cf_serve_wait(sv, t, 30_000_000) for t in tickets]
    for t in tickets:
        cf.cf_serve_release(sv, t)
    return res, outs, t_first


def test_served_fields_match_cf_sample():
    sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=3))
    res, outs, _ = _serve(sv, REQS)
    for (n, kind, amp, scale, beta, seed, r0, R), r, (hf, _) in zip(REQS, res, outs):
        assert r["status"] == cf.CF_OK
        emb = cf.cf_embed(cf.make_grid(n), cf.make_xi(kind, amp, scale, beta), cf.CF_EMBED_CLAMP)
        wsb = cf.cf_sample_workspace_size(emb, R, cf.CF_F32)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=DEV)
        ref = torch.empty((R, 2) + n, dtype=torch.float32, device=DEV)
        cf.cf_sample(emb, seed, r0, R, cf.CF_F32, ref, ws, wsb)
        torch.cuda.synchronize()
        ref = ref.cpu().double().numpy()
        got = hf.double().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        assert r["embed"]["lambda_max"] == pytest.approx(emb.report["lambda_max"], rel=1e-9)
        emb.close()
    st = cf.cf_serve_stats(sv)
    assert st["completed"] == len(REQS) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    cf.cf_serve_destroy(sv)


def test_same_result_alone_and_in_a_mixed_batched_stream():
    rng = np.random.default_rng(3)
    specs = []
    for i in range(40):
        n, kind, amp, scale, beta, seed, r0, R = REQS[i % len(REQS)]
        specs.append((n, kind, float(rng.uniform(0.2, 1.5)), scale, beta, 1000 + i, int(rng.integers(0, 50)),
                      int(rng.integers(1, 5))))
    alone_sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=1, max_batch_realizations=8))
    alone = []
    for s in specs[:12]:
        _, outs, _ = _serve(alone_sv, [s], want_counts=True)
        alone.append(outs[0])
    cf.cf_serve_destroy(alone_sv)
    # one slot, held by a large request while the mixed stream queues behind
    # it, so that the queued requests of each shape are batched
    mix_sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=1, max_batch_realizations=64))
    big = cf.make_request((1024, 1024), cf.CF_XI_GAUSSIAN, 1.0, 4.0, R=64)
    res, outs, blocker = _serve(mix_sv, specs, want_counts=True, first=big)
    assert cf.cf_serve_wait(mix_sv, blocker, 30_000_000)["status"] == cf.CF_OK
    cf.cf_serve_release(mix_sv, blocker)
    st = cf.cf_serve_stats(mix_sv)
    assert all(r["status"] == cf.CF_OK for r in res)
    assert st["batches"] < st["batched_requests"]  # requests were batched
    assert st["cache_hits"] > 0
    for (fa, ca), (fm, cm) in zip(alone, outs[:12]):
        assert torch.equal(fa, fm)
        assert torch.equal(ca, cm)
    cf.cf_serve_destroy(mix_sv)


def test_served_counts_match_standalone_poisson():
    sv = cf.cf_serve_create(cf.make_serve_cfg())
    spec = ((64, 64), cf.CF_XI_GAUSSIAN, 0.8, 3.0, 0.0, 21, 4, 3)
    res, outs, _ = _serve(sv, [spec], want_counts=True)
    hf, hc = outs[0]
    f = hf.to(DEV)
    c = torch.empty(hc.shape, dtype=torch.int32, device=DEV)
    cf.cf_lognormal_poisson(f, cf.CF_F32, 64 * 64, 2 * 3, 0.8, 2.0, None, 22, 2 * 4, None, c)
    torch.cuda.synchronize()
    assert torch.equal(c.cpu(), hc)
    cf.cf_serve_destroy(sv)


def test_failures_are_statuses():
    sv = cf.cf_serve_create(cf.make_serve_cfg(hbm_budget=64 << 20))
    t1 = cf.cf_serve_submit(sv, cf.make_request((64, 64), cf.CF_XI_GEN_CAUCHY, 0.8, 8.0, 0.4, R=1, embed_flags=0))
    t2 = cf.cf_serve_submit(sv, cf.make_request((1024, 1024), cf.CF_XI_GAUSSIAN, 1.0, 4.0, R=32))
    t3 = cf.cf_serve_submit(sv, cf.make_request((32, 32), cf.CF_XI_GAUSSIAN, 1.0, 2.0, R=1))
    r1 = cf.cf_serve_wait(sv, t1, 30_000_000)
    r2 = cf.cf_serve_wait(sv, t2, 30_000_000)
    r3 = cf.cf_serve_wait(sv, t3, 30_000_000)
    assert r1["status"] == cf.CF_ERR_NOT_PSD and r1["embed"]["n_negative"] > 0
    assert r2["status"] == cf.CF_ERR_NOMEM
    assert r3["status"] == cf.CF_OK
    with pytest.raises(cf.CfError) as ei:
        cf.cf_serve_submit(sv, cf.make_request((32, 32), cf.CF_XI_GAUSSIAN, -1.0, 2.0, R=1))
    assert ei.value.status == cf.CF_ERR_ARG
    for t in (t1, t2, t3):
        cf.cf_serve_release(sv, t)
    st = cf.cf_serve_stats(sv)
    assert st["failed"] == 2 and st["completed"] == 1
    cf.cf_serve_destroy(sv)


def test_batched_mixed_stream_matches_the_oracle(orc):
    """Requests of one shape queued behind a large one are served by one
    descriptor-driven launch (different amplitude, seed, realization offset
    and Poisson parameters per request); every served field is compared with
    the oracle's sampler at the request's amplitude (binary32 gate, relative
    L2 1e-5) and every count with the oracle's inverse CDF on the served
    field (bit-exact outside the 1e-6 boundary band)."""
    specs = [((64, 64), cf.CF_XI_GAUSSIAN, 0.35, 3.0, 0.0, 501, 0, 3, 0.35, 2.0),
             ((64, 64), cf.CF_XI_GAUSSIAN, 1.20, 3.0, 0.0, 502, 17, 2, 1.20, 5.0),
             ((64, 64), cf.CF_XI_GAUSSIAN, 0.80, 3.0, 0.0, 0xABCDEF0123, 2**32 - 9, 4, 0.80, 0.5),
             ((16, 16, 16), cf.CF_XI_EXPONENTIAL, 0.9, 2.0, 0.0, 504, 3, 2, 0.9, 3.0),
             ((16, 16, 16), cf.CF_XI_EXPONENTIAL, 0.4, 2.0, 0.0, 505, 9, 3, 0.4, 1.0),
             ((64, 64), cf.CF_XI_GEN_CAUCHY, 0.6, 4.0, 0.4, 506, 1, 2, 0.6, 2.0),
             # rows of 1024 points (the warp row pass with descriptors)
             ((512, 512), cf.CF_XI_GEN_CAUCHY, 0.8, 8.0, 0.4, 507, 4, 2, 0.8, 2.0),
             ((512, 512), cf.CF_XI_GEN_CAUCHY, 0.5, 8.0, 0.4, 508, 0, 1, 0.5, 1.0)]
    sv = cf.cf_serve_create(cf.make_serve_cfg(max_inflight=1, max_batch_realizations=64))
    big = cf.make_request((1024, 1024), cf.CF_XI_GAUSSIAN, 1.0, 4.0, R=64)
    t_big = cf.cf_serve_submit(sv, big)
    tickets, outs, keep = [], [], []
    for n, kind, amp, scale, beta, seed, r0, R, s2, nbar in specs:
        hf, hc = _host((R, 2) + n), _host((R, 2) + n, torch.int32)
        req = cf.make_request(n, kind, amp, scale, beta, seed=seed, r0=r0, R=R, want_counts=True, sigma2=s2,
                              nbar=nbar, lp_seed=seed + 7, host_fields=hf, host_counts=hc)
        keep.append(req)
        tickets.append(cf.cf_serve_submit(sv, req))
        outs.append((hf, hc))
    res = [cf.cf_serve_wait(sv, t, 60_000_000) for t in tickets]
    assert cf.cf_serve_wait(sv, t_big, 60_000_000)["status"] == cf.CF_OK
    st = cf.cf_serve_stats(sv)
    assert st["batches"] < st["batched_requests"], "the queued requests were not batched"
    for (n, kind, amp, scale, beta, seed, r0, R, s2, nbar), r, (hf, hc) in zip(specs, res, outs):
        assert r["status"] == cf.CF_OK
        o = orc.embed(list(n), kind, amp, scale, beta, clamp=True)
        ref = orc.sample(n, o["sqrt_lambda"], seed, r0, R, 1)
        got = hf.double().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (n, amp, seed, err)
        _, oc, margin = orc.lognormal_poisson(got.reshape(2 * R, -1), s2, nbar, seed=seed + 7, field0=2 * r0)
        c = hc.numpy().reshape(2 * R, -1)
        bad = (c != oc) & (margin >= 1e-6)
        assert not bad.any(), (n, seed, int(bad.sum()))
        assert (margin < 1e-6).mean() < 1e-3
    for t in tickets + [t_big]:
        cf.cf_serve_release(sv, t)
    cf.cf_serve_destroy(sv)
