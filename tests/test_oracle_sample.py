"""Pins for the oracle's per-realization Gaussian fields (section 2, CPU only).

* Exactness, the paper's central claim (eq. (thatiswhatwewant) and the
  closing paragraph of section 2): the sampler is a linear map W = A eps of
  the complex noise; its covariance Re(A A^H) on the survey box must equal
  xi(x - y) for every pair of cells, and Im(A A^H) (the Re/Im cross
  covariance) must vanish.  Checked to round-off on rectangular 2D and 3D
  grids by feeding the map basis vectors.
* The sample covariance over many realizations converges to xi within a CLT
  band, with both noise precisions.
* Brute-force Cholesky sampling of the N^d x N^d target gives statistically
  identical fields (two-sample KS tests on linear functionals).
"""
import numpy as np
import pytest
from scipy import stats


def _target_cov(n, c):
    """Survey covariance matrix xi(x - y) read off the embedded row c."""
    M = c.shape
    idx = np.indices(n).reshape(len(n), -1).T
    C = np.empty((idx.shape[0],) * 2)
    for a, x in enumerate(idx):
        d = (x[None, :] - idx) % np.asarray(M)
        C[a] = c[tuple(d.T)]
    return C


def _linear_map(orc, n, s):
    total = int(np.asarray(s).size)
    cols = []
    for k in range(total):
        e = np.zeros(total, dtype=np.complex128)
        e[k] = 1.0
        cols.append(orc.sample_given_noise(n, s, e).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("n,kind,scale", [((4, 6), 0, 0.7), ((3, 4, 2), 2, 0.7), ((8,), 0, 1.5),
                                          ((5, 3), 0, 0.4)])
def test_sampler_is_exact_on_the_survey(orc, n, kind, scale):
    e = orc.embed(list(n), kind, 1.1, scale, 0.4)
    assert e["report"]["status"] == 0 and e["report"]["clamped"] == 0
    A = _linear_map(orc, n, e["sqrt_lambda"])
    AAH = A @ A.conj().T
    C = _target_cov(n, e["c"])
    assert np.max(np.abs(AAH.real - C)) < 1e-12 * C.max()
    assert np.max(np.abs(AAH.imag)) < 1e-12 * C.max()
    # A A^T = 0 is automatic for complex noise; W W^T has zero expectation
    # The two fields are uncorrelated: E[Re W Im W^T] = -Im(A A^H) = 0 (above).


@pytest.mark.parametrize("n,M,kind,scale", [((4, 3), (16, 12), 0, 0.7), ((3, 2, 2), (24, 16, 16), 2, 0.9),
                                            ((6,), (48,), 0, 1.2), ((3, 5), (8, 16), 2, 0.8), ((5,), (16,), 0, 0.9)])
def test_padded_sampler_is_exact_on_the_survey(orc, n, M, kind, scale):
    """On a periodic grid of M_i >= 2 n_i points the survey box is still a
    sub-box of side at most half the period, so its covariance Re(A A^H) is
    xi(x - y) exactly: compared with xi evaluated in closed form at the cell
    separations (not read off the oracle's own row).  Covers p times the side
    and survey sizes embedded in the next power of two."""
    e = orc.embed(list(n), kind, 1.1, scale, 0.0, M=M)
    assert e["report"]["status"] == 0 and e["report"]["clamped"] == 0
    A = _linear_map(orc, n, e["sqrt_lambda"])
    AAH = A @ A.conj().T
    idx = np.indices(n).reshape(len(n), -1).T
    r = np.sqrt(((idx[:, None, :] - idx[None, :, :]) ** 2).sum(-1))
    C = 1.1 * (np.exp(-r**2 / (2 * scale**2)) if kind == 0 else np.exp(-r / scale))
    assert np.max(np.abs(AAH.real - C)) < 1e-12 * C.max()
    assert np.max(np.abs(AAH.imag)) < 1e-12 * C.max()


def test_clamped_sampler_realises_inverse_transform_of_lambda_plus(orc):
    n = (8, 8)
    e = orc.embed(list(n), 1, 0.8, 4.0, 0.4, clamp=True)
    assert e["report"]["clamped"] == 1
    A = _linear_map(orc, n, e["sqrt_lambda"])
    realised = np.real(np.fft.ifftn(e["lambda_plus"]))
    C = _target_cov(n, realised)
    assert np.max(np.abs((A @ A.conj().T).real - C)) < 1e-12
    assert np.max(np.abs(C - _target_cov(n, e["c"]))) == pytest.approx(e["report"]["cov_error"],
                                                                       rel=1e-6)


def test_sample_is_noise_then_map(orc):
    n = (4, 8)
    e = orc.embed(list(n), 0, 1.0, 0.7, 0)
    for dtype in (0, 1):
        f = orc.sample(n, e["sqrt_lambda"], 9, 5, 2, dtype)
        eps = orc.draw_noise(9, 5, 2, 8 * 16, 16, dtype)
        for r in range(2):
            w = orc.sample_given_noise(n, e["sqrt_lambda"], eps[r])
            assert np.array_equal(f[r, 0], w.real) and np.array_equal(f[r, 1], w.imag)


@pytest.mark.parametrize("dtype", [0, 1])
def test_sample_covariance_converges(orc, dtype):
    n = (4, 4)
    e = orc.embed(list(n), 0, 1.0, 0.7, 0)
    assert e["report"]["status"] == 0
    R = 20000
    f = orc.sample(n, e["sqrt_lambda"], 31 + dtype, 0, R, dtype)
    X = f.reshape(R * 2, -1)          # Re and Im fields are independent draws
    Chat = np.cov(X, rowvar=False, bias=True) + np.outer(X.mean(0), X.mean(0))
    C = _target_cov(n, e["c"])
    sig = np.sqrt((np.outer(np.diag(C), np.diag(C)) + C**2) / X.shape[0])
    assert np.max(np.abs(Chat - C) / sig) < 6.0
    assert np.max(np.abs(X.mean(0)) / np.sqrt(np.diag(C) / X.shape[0])) < 6.0
    # Re/Im cross covariance
    re = f[:, 0].reshape(R, -1)
    im = f[:, 1].reshape(R, -1)
    cross = re.T @ im / R
    sigx = np.sqrt(np.outer(np.diag(C), np.diag(C)) / R)
    assert np.max(np.abs(cross) / sigx) < 6.0


def test_matches_cholesky_sampling(orc):
    """Brute-force exact sampling by Cholesky factorisation of the survey
    covariance (cost >= N_cells^2, the paper's section 1 comparison)."""
    n = (6, 6)
    e = orc.embed(list(n), 0, 1.0, 1.0, 0)
    assert e["report"]["status"] == 0
    C = _target_cov(n, e["c"])
    L = np.linalg.cholesky(C + 1e-13 * np.eye(C.shape[0]))
    R = 6000
    rng = np.random.default_rng(44)
    chol = (L @ rng.standard_normal((C.shape[0], 2 * R))).T
    f = orc.sample(n, e["sqrt_lambda"], 45, 0, R, 0).reshape(2 * R, -1)
    w_sum = np.ones(C.shape[0])
    w_grad = np.tile(np.arange(n[1]) - 2.5, n[0])
    w_corner = np.zeros(C.shape[0])
    w_corner[0], w_corner[-1] = 1.0, -1.0
    for w in (w_sum, w_grad, w_corner):
        a, b = f @ w, chol @ w
        assert stats.ks_2samp(a, b).pvalue > 1e-3
        # both match the analytic variance w^T C w
        v = w @ C @ w
        for x in (a, b):
            assert abs(x.var() / v - 1) < 6 * np.sqrt(2 / x.size)
