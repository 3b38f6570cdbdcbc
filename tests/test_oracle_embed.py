"""Pins for the oracle's transforms and circulant embedding (section 2, CPU only).

* naive DFT and recursive FFT against numpy.fft (an independent library) and
  against each other;
* the embedded first row against the lag rule of eq. (grid) (index n on an
  axis of size 2n carries lag -n) and the closed-form xi families;
* lambda against a direct O(M^{2d}) sum written with explicit exponentials,
  against the closed form of a delta row (lambda == 1), and through the
  inverse-transform round trip (the circulant is diagonalised exactly);
* the positivity check on strictly positive and on non-PSD families, with the
  clamped covariance error recomputed independently.
"""
import numpy as np
import pytest

from paper_1406_6072_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 12])
def test_naive_dft_matches_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(orc.dft_naive(x, -1), np.fft.fft(x), atol=1e-12)
    assert np.allclose(orc.dft_naive(x, +1), np.fft.ifft(x) * n, atol=1e-12)


@pytest.mark.parametrize("n", [2, 4, 32, 64, 1024, 4096])
def test_recursive_fft_matches_numpy(orc, n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    got = orc.fft_recursive(x, -1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.sqrt(n) * np.max(np.abs(ref))
    back = orc.fft_recursive(got, +1) / n
    assert np.max(np.abs(back - x)) < 1e-13
    if n <= 64:
        assert np.allclose(orc.dft_naive(x, -1), got, atol=1e-12)


@pytest.mark.parametrize("shape", [(8,), (16, 32), (6, 10), (4, 8, 16), (64, 32)])
def test_fft_nd_matches_numpy(orc, shape):
    rng = np.random.default_rng(len(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.allclose(orc.fft_nd(x, -1), np.fft.fftn(x), atol=1e-10)
    assert np.allclose(orc.fft_nd(x, +1), np.fft.ifftn(x) * x.size, atol=1e-10)


def _xi(kind, r, amp, scale, beta):
    if kind == 0:
        return amp * np.exp(-r**2 / (2 * scale**2))
    if kind == 1:
        return amp / (1 + (r / scale) ** 2) ** beta
    return amp * np.exp(-r / scale)


@pytest.mark.parametrize("kind,amp,scale,beta", [(0, 1.0, 4.0, 0), (1, 0.8, 8.0, 0.4), (2, 1.0, 6.0, 0)])
def test_embedded_row_lag_rule(orc, kind, amp, scale, beta):
    n = [4, 6]
    c = orc.embed_row(n, kind, amp, scale, beta, cell=[1.5, 0.5])
    assert c.shape == (8, 12)
    for i in range(8):
        for j in range(12):
            li = i if i < 4 else i - 8
            lj = j if j < 6 else j - 12
            r = np.hypot(li * 1.5, lj * 0.5)
            assert c[i, j] == pytest.approx(_xi(kind, r, amp, scale, beta), rel=1e-14)
    # index n carries lag -n, so the row is symmetric under m -> -m mod M
    assert np.array_equal(c, np.roll(c[::-1, ::-1], (1, 1), axis=(0, 1)))


def _direct_dft_real(c):
    """lambda_k = sum_m c_m exp(-2 pi i k.m/M) as an explicit double sum."""
    dims = c.shape
    idx = np.indices(dims).reshape(len(dims), -1).T
    lam = np.zeros(c.size, dtype=np.complex128)
    flat = c.ravel()
    for a, k in enumerate(idx):
        phase = np.zeros(len(idx))
        for d, M in enumerate(dims):
            phase += (k[d] * idx[:, d] % M) / M
        lam[a] = np.sum(flat * np.exp(-2j * np.pi * phase))
    return lam.reshape(dims)


@pytest.mark.parametrize("n,kind", [([8], 0), ([4, 6], 1), ([8, 8], 0), ([4, 4, 4], 2), ([3, 5], 2)])
def test_lambda_direct_dft_and_round_trip(orc, n, kind):
    c = orc.embed_row(n, kind, 0.9, 2.5, 0.4)
    lam = orc.eigenvalues(n, c)
    direct = _direct_dft_real(c)
    assert np.max(np.abs(lam - direct.real)) <= 1e-13 * np.sum(np.abs(c))
    assert np.max(np.abs(direct.imag)) <= 1e-12 * np.sum(np.abs(c))
    # the circulant is diagonalised: inverse transform of lambda returns c
    back = np.real(orc.fft_nd(lam.astype(np.complex128), +1)) / lam.size
    assert np.max(np.abs(back - c)) <= 1e-13 * np.max(np.abs(c))


def test_delta_row_has_unit_spectrum(orc):
    n = [16]
    table = np.zeros(32)
    table[0] = 1.0
    c = orc.embed_row(n, orc.XI_TABLE, table=table)
    assert np.allclose(orc.eigenvalues(n, c), 1.0, atol=1e-15)
    n2 = [4, 8]
    t2 = np.zeros((8, 16))
    t2[0, 0] = 2.0
    assert np.allclose(orc.eigenvalues(n2, orc.embed_row(n2, 3, table=t2)), 2.0, atol=1e-15)


def test_circulant_eigen_decomposition(orc):
    """The full M^d x M^d covariance built from c has eigenvalues lambda
    (the circulant picture of the paper's first figure)."""
    n = [3, 4]
    c = orc.embed_row(n, 0, 1.0, 1.2, 0)
    M = c.shape
    idx = np.indices(M).reshape(2, -1).T
    cov = np.empty((idx.shape[0],) * 2)
    for a, x in enumerate(idx):
        for b, y in enumerate(idx):
            cov[a, b] = c[(x[0] - y[0]) % M[0], (x[1] - y[1]) % M[1]]
    ev = np.sort(np.linalg.eigvalsh(cov))
    lam = np.sort(orc.eigenvalues(n, c).ravel())
    assert np.allclose(ev, lam, atol=1e-12)


def test_exponential_family_is_strictly_positive(orc):
    """exp(-r/6) on a 128^3 survey embeds exactly; checked here at the same
    scale-to-survey ratio on 32^3 (scale 1.5).  With the scale as large as a
    quarter of the survey (16^3, scale 6) the same family is not PSD."""
    cfg = W.CONFIGS["exp3d_n128"]
    n = [32, 32, 32]
    e = orc.embed(n, cfg.xi_kind, cfg.amp, cfg.scale * 32 / cfg.n[0], cfg.beta)
    assert orc.embed([16] * 3, cfg.xi_kind, cfg.amp, cfg.scale, 0)["report"]["status"] == 2
    assert e["report"]["lambda_min"] > 0
    assert e["report"]["status"] == 0 and e["report"]["clamped"] == 0
    assert e["report"]["n_negative"] == 0


def test_gaussian_family_psd_to_roundoff(orc):
    cfg = W.CONFIGS["gauss2d_n64_f64"]
    e = orc.embed(cfg.n, cfg.xi_kind, cfg.amp, cfg.scale, cfg.beta)
    rep = e["report"]
    assert rep["status"] == 0 and rep["n_negative"] == 0
    assert rep["lambda_min"] / rep["lambda_max"] > -1e-12
    assert np.all(e["sqrt_lambda"] ** 2 == e["lambda_plus"]) or np.allclose(
        e["sqrt_lambda"] ** 2, e["lambda_plus"], rtol=1e-15, atol=0)


def test_non_psd_family_fails_then_clamps(orc):
    """The generalised-Cauchy family with a slow r^-0.8 tail is not PSD on a
    doubled grid; without clamping the embedding reports failure (the paper's
    'the method fails'), with clamping it reports the realised error."""
    cfg = W.CONFIGS["cauchy2d_n512_f32"]
    n = [64, 64]
    c = orc.embed_row(n, cfg.xi_kind, cfg.amp, cfg.scale, cfg.beta)
    lam = orc.eigenvalues(n, c)
    lp, s, rep = orc.psd(n, c, lam, clamp=False)
    assert lam.min() < -1e-12 * lam.max()
    assert rep["status"] == 2 and rep["n_negative"] > 0
    lp, s, rep = orc.psd(n, c, lam, clamp=True)
    assert rep["status"] == 0 and rep["clamped"] == 1
    assert np.all(lp >= 0) and np.all(s >= 0)
    # independent recomputation of the realised covariance error (numpy ifft)
    real_cov = np.real(np.fft.ifftn(lp))
    mask = np.ones(c.shape, bool)
    mask[n[0], :] = False
    mask[:, n[1]] = False
    err = np.max(np.abs(real_cov - c)[mask])
    assert rep["cov_error"] == pytest.approx(err, rel=1e-9)
    assert 0 < rep["cov_error"] < 1e-2  # 1.8e-3 at 64^2; 3.1e-5 at 512^2
    assert rep["neg_mass"] == pytest.approx(-lam[lam < -rep["tau"]].sum(), rel=1e-12)


def test_threshold_zeroes_tiny_eigenvalues(orc):
    n = [4]
    lam = np.array([10.0, 1e-12, -1e-12, 5e-11, -5e-11, 3.0, 0.0, 2.0])
    c = np.real(np.fft.ifft(lam))
    lp, s, rep = orc.psd(n, c, lam, clamp=False)
    # tau = 1e-11: +-1e-12 and 0 zeroed; +5e-11 kept; -5e-11 negative -> failure
    assert rep["tau"] == pytest.approx(1e-11)
    assert rep["status"] == 2 and rep["n_negative"] == 1 and rep["n_zeroed"] == 3
    lp, s, rep = orc.psd(n, c, lam, clamp=True)
    assert list(lp) == [10.0, 0.0, 0.0, 5e-11, 0.0, 3.0, 0.0, 2.0]
    assert np.array_equal(s, np.sqrt(lp))


@pytest.mark.parametrize("box_factor", [1, 2, 4])
def test_periodic_box_spectrum_matches_continuous_transform(orc, box_factor):
    """Section 3.3, eq. (Periodicboxmodes): for the Gaussian family the
    continuous spectrum is P(k) = amp 2 pi s^2 exp(-k^2 s^2 / 2) (2D); the box
    modes k = 2 pi m / B carry it, the DC mode is zero, and for box_factor 1
    the modes sit on the even frequencies of the 2n grid with weight 4."""
    n, s, amp = (32, 32), 3.0, 0.7
    lam = orc.periodic_lambda(n, 0, amp, s, 0.0, box_factor, 2, 4)
    Me = lam.shape
    B = [(v // 2 if box_factor == 1 else v) for v in Me]
    idx = np.indices(Me)
    k2 = np.zeros(Me)
    on = np.ones(Me, dtype=bool)
    for a in range(2):
        m = idx[a]
        if box_factor == 1:
            on &= m % 2 == 0
            m = m // 2
        f = np.where(m < B[a] // 2, m, m - B[a])
        k2 = k2 + (2 * np.pi * f / B[a]) ** 2
    P = amp * 2 * np.pi * s * s * np.exp(-k2 * s * s / 2) * (4.0 if box_factor == 1 else 1.0)
    P[~on] = 0.0
    P[0, 0] = 0.0
    assert np.max(np.abs(lam - P)) <= 1e-12 * P.max()


# ---------------------------------------------------------------- larger embedding grids
def _xi_closed_form(kind, amp, scale, beta, r):
    if kind == 0:
        return amp * np.exp(-r**2 / (2 * scale**2))
    if kind == 1:
        return amp * (1 + (r / scale) ** 2) ** (-beta)
    return amp * np.exp(-r / scale)


@pytest.mark.parametrize("n,p,kind", [([4], 4, 0), ([4], 8, 2), ([2, 3], 4, 1), ([2, 2, 1], 8, 0)])
def test_padded_row_lags_and_spectrum(orc, n, p, kind):
    """Embedding on p times the survey side: index m_i has lag m_i below M_i/2
    and m_i - M_i from M_i/2 on (for p = 2 the paper's grid -n..n-1); the
    eigenvalues are the row's DFT (direct sum)."""
    c = orc.embed_row(n, kind, 0.9, 1.7, 0.4, factor=p)
    M = tuple(p * v for v in n)
    assert c.shape == M
    for idx in np.ndindex(*M):
        lag = np.array([m if 2 * m < Mi else m - Mi for m, Mi in zip(idx, M)], dtype=np.float64)
        assert c[idx] == pytest.approx(_xi_closed_form(kind, 0.9, 1.7, 0.4, np.sqrt(np.sum(lag**2))), rel=1e-15)
    lam = orc.eigenvalues(n, c)
    direct = _direct_dft_real(c)
    assert np.max(np.abs(lam - direct.real)) <= 1e-13 * np.sum(np.abs(c))


def test_padding_reduces_the_clamping_error(orc):
    """Wood and Chan's remedy, cited in section 1: a larger periodic grid
    makes the embedded spectrum less negative.  For the slowly decaying
    generalised Cauchy family (not PSD on any of these grids) the clamped
    covariance error falls about fourfold per doubling of the grid."""
    errs = []
    for p in (2, 4, 8):
        e = orc.embed([16, 16], 1, 0.8, 2.0, 0.4, clamp=True, factor=p)
        assert e["report"]["clamped"] == 1
        errs.append(e["report"]["cov_error"])
        # the reported error is that of the realised covariance IDFT(lambda+)
        realised = np.real(np.fft.ifftn(e["lambda_plus"]))
        M = e["c"].shape
        survey = np.ix_(*[np.r_[0:16, M[a] - 15:M[a]] for a in range(2)])
        assert np.max(np.abs(realised - e["c"])[survey]) == pytest.approx(e["report"]["cov_error"], rel=1e-9)
    assert errs[1] < errs[0] / 2 and errs[2] < errs[1] / 2
