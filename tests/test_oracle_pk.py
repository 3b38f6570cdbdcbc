"""Pins for the oracle's binned power spectrum (section 3.2, eq. (Def spec))
and its mean/covariance over realizations (CPU only).

* brute force: explicit DFT sums and explicit binning on tiny 2D/3D grids;
* Parseval's identity with one all-covering bin;
* white noise has flat expected power cell^d sigma^2;
* the exact sampler's expected periodogram equals the Fejer-weighted
  covariance sum_r prod(N - |r_i|) xi(r) e^{-i k.r} (closed form);
* the paper's Gaussian information limit (section 3.3): I(<= l) equals half
  the number of modes for a Gaussian field with independent modes;
* delta_g of eq. (Estim): sum_i f_i delta_g,i = 0, zero on masked cells;
* mean and unbiased covariance against numpy.
"""
import math

import numpy as np
import pytest

from paper_1406_6072_gb300 import workloads as W


def _mode_lengths(n, cell):
    """|k| of every mode of an n-grid with cell sizes `cell`, in units of the
    fundamental 2 pi / L_ref of the longest side L_ref = max n_d cell_d,
    computed directly from k_d = s_d / (n_d cell_d) (cycles per unit)."""
    d = len(n)
    cell = np.broadcast_to(np.asarray(cell, dtype=np.float64), (d,))
    L = np.array(n, dtype=np.float64) * cell
    idx = np.indices(n).reshape(d, -1).T
    s = np.where(2 * idx <= np.array(n), idx, idx - np.array(n))
    return L.max() * np.sqrt(np.sum((s / L) ** 2, axis=1))


def _brute_pk(field, edges, cell):
    n = field.shape
    d = len(n)
    cellv = np.broadcast_to(np.asarray(cell, dtype=np.float64), (d,))
    idx = np.indices(n).reshape(d, -1).T
    flat = field.ravel()
    nb = edges.size - 1
    sums = np.zeros(nb)
    counts = np.zeros(nb, dtype=np.int64)
    q = _mode_lengths(n, cellv)
    for t, k in enumerate(idx):
        ph = np.zeros(len(idx))
        for a in range(d):
            ph += (k[a] * idx[:, a] % n[a]) / n[a]
        X = np.sum(flat * np.exp(-2j * np.pi * ph))
        if not np.any(k):
            continue
        kn = q[t]
        for b in range(nb):
            if edges[b] <= kn < edges[b + 1]:
                sums[b] += abs(X) ** 2
                counts[b] += 1
    pk = np.where(counts > 0, np.prod(cellv) * sums / (np.prod(n) * np.maximum(counts, 1)), 0.0)
    return pk, counts


@pytest.mark.parametrize("n,cell", [((6, 8), 1.0), ((4, 4, 4), 0.5), ((12,), 2.0), ((8, 8), 1.0),
                                    ((5, 4, 3), (0.5, 0.7, 1.1)), ((6, 10), (2.0, 1.0)), ((9, 7), 1.0)])
def test_power_spectrum_brute_force(orc, n, cell):
    rng = np.random.default_rng(sum(n))
    fields = rng.standard_normal((3,) + n)
    q = _mode_lengths(n, cell)
    cube = len(set(n)) == 1 and np.ndim(cell) == 0
    # cubes: integer edges (exact integer mode lengths); otherwise edges that
    # no mode length comes near, so that rounding cannot decide a bin
    kmax = q.max() * 0.9 if not cube else min(n) / 2
    edges = orc.bin_edges(orc.BINS_LINEAR, 3, 0.0, kmax if cube else kmax + 0.0123)
    if not cube:
        assert np.min(np.abs(q[q > 0][:, None] - edges[None, :])) > 1e-9
    pk, nm = orc.power_spectrum(fields, n, edges, cell=cell)
    for f in range(3):
        ref, cnt = _brute_pk(fields[f], edges, cell)
        assert np.array_equal(nm, cnt)
        assert np.allclose(pk[f], ref, rtol=1e-11, atol=1e-13)


def test_power_spectrum_plane_waves_in_a_rectangular_box(orc):
    """A plane wave of physical wavelength lam puts all its power at
    |k| = L_ref / lam (fundamental units of the longest side), whatever the
    axis and cell size: box 10 x 6 cells of 1 x 2 units (L = 10, 12)."""
    n, cell = (10, 6), (1.0, 2.0)
    i0, i1 = np.indices(n)
    waves = {2.4: np.cos(2 * np.pi * 2 * i0 / 10),      # wavelength 5 units along axis 0
             1.0: np.cos(2 * np.pi * 1 * i1 / 6),       # wavelength 12 units along axis 1
             3.0: np.cos(2 * np.pi * 3 * i1 / 6)}       # wavelength 4 units along axis 1 (Nyquist)
    edges = np.array([0.5, 1.5, 2.7, 3.5])
    for q, f in waves.items():
        pk, nm = orc.power_spectrum(f[None], n, edges, cell=cell)
        hit = np.searchsorted(edges, q, side="right") - 1
        assert pk[0, hit] > 0
        assert np.all(pk[0, np.arange(3) != hit] < 1e-20 * pk[0, hit])


def test_parseval(orc):
    rng = np.random.default_rng(1)
    n = (16, 32)
    x = rng.standard_normal((2,) + n)
    pk, nm = orc.power_spectrum(x, n, np.array([0.0, 1e9]))
    assert nm[0] == 16 * 32 - 1
    for f in range(2):
        total = pk[f, 0] * nm[0] * x[f].size  # sum over k != 0 of |X_k|^2
        assert total == pytest.approx(x[f].size * np.sum(x[f] ** 2) - np.sum(x[f]) ** 2, rel=1e-12)


def test_white_noise_is_flat(orc):
    n = (32, 32)
    x = W.gaussian_field_values((200,) + n, seed=2, scale=1.5)
    edges = orc.bin_edges(orc.BINS_LINEAR, 8, 0.0, 16.0)
    pk, nm = orc.power_spectrum(x, n, edges, cell=2.0)
    mean = pk.mean(0)
    expect = 4.0 * 2.25  # cell^2 sigma^2
    sig = expect * np.sqrt(2.0 / (nm * 200))
    assert np.all(np.abs(mean - expect) < 6 * sig)


def test_expected_periodogram_of_exact_fields(orc):
    """E|DFT G|^2 at k = sum over lags r with |r_i| < N of prod_i(N-|r_i|)
    xi(r) e^{-i k.r}: one FFT of the Fejer-weighted row on the 2N grid."""
    n = (16, 16)
    e = orc.embed(list(n), 0, 1.0, 1.2, 0)
    assert e["report"]["status"] == 0
    c = e["c"]
    M = c.shape
    lag = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in M]
    wgt = np.outer(np.where(np.abs(lag[0]) < n[0], n[0] - np.abs(lag[0]), 0),
                   np.where(np.abs(lag[1]) < n[1], n[1] - np.abs(lag[1]), 0))
    expect_full = np.real(np.fft.fft2(wgt * c))[::2, ::2]  # k = 2 pi j / N
    edges = orc.bin_edges(orc.BINS_LINEAR, 4, 0.0, 8.0)
    # bin the expectation with the same rule
    sums = np.zeros(4)
    cnt = np.zeros(4)
    for i in range(16):
        for j in range(16):
            si = i if i <= 8 else i - 16
            sj = j if j <= 8 else j - 16
            k2 = si * si + sj * sj
            if k2 == 0:
                continue
            kn = math.sqrt(k2)
            for b in range(4):
                if edges[b] <= kn < edges[b + 1]:
                    sums[b] += expect_full[i, j]
                    cnt[b] += 1
    expect = sums / (cnt * 256)
    R = 1500
    fields = orc.sample(n, e["sqrt_lambda"], 3, 0, R, 0).reshape(2 * R, *n)
    pk, nm = orc.power_spectrum(fields, n, edges)
    assert np.array_equal(nm, cnt)
    mean = pk.mean(0)
    sd = pk.std(0) / np.sqrt(2 * R)
    assert np.all(np.abs(mean - expect) < 6 * sd), (mean, expect, sd)


def test_gaussian_information_is_half_the_modes(orc):
    """Section 3.3: for Gaussian statistics I(<= l) = sum C^{-1} is half the
    number of modes below l, C = <P P>/(<P><P>) - 1."""
    n = (16, 16)
    x = W.gaussian_field_values((4000,) + n, seed=3)
    edges = orc.bin_edges(orc.BINS_LINEAR, 4, 0.0, 8.0)
    pk, nm = orc.power_spectrum(x, n, edges)
    mean, cov = orc.mean_cov(pk)
    C = cov / np.outer(mean, mean)
    info = np.linalg.inv(C).sum()
    assert info == pytest.approx(nm.sum() / 2, rel=0.08)
    cum = orc.cumulative_information(mean, cov)
    assert cum[-1] == pytest.approx(info, rel=1e-12)
    assert np.allclose(cum, np.cumsum(nm) / 2, rtol=0.1)


def test_cumulative_information_closed_forms(orc):
    """Eq. (cuminfo) on matrices with a known inverse: diagonal C gives the
    running sum of 1/C_bb; a 2 x 2 block [[a, c], [c, d]] gives
    (a + d - 2c) / (ad - c^2); a bin with zero mean is skipped."""
    mean = np.array([2.0, 0.0, 1.0, 4.0])
    cdiag = np.array([0.5, 1.0, 0.25, 0.125])
    cov = np.diag(cdiag) * np.outer(mean, mean)
    cum = orc.cumulative_information(mean, cov)
    assert np.allclose(cum, [2.0, 2.0, 6.0, 14.0], rtol=1e-13)
    a, c, d = 0.4, 0.1, 0.3
    m2 = np.array([3.0, 5.0])
    cov2 = np.array([[a, c], [c, d]]) * np.outer(m2, m2)
    cum2 = orc.cumulative_information(m2, cov2)
    assert cum2[0] == pytest.approx(1 / a, rel=1e-13)
    assert cum2[1] == pytest.approx((a + d - 2 * c) / (a * d - c * c), rel=1e-13)


def test_counts_to_delta(orc):
    f = W.survey_mask((16, 16), seed=4).ravel().astype(np.float64)
    counts = np.random.default_rng(5).poisson(3.0 * f, size=(3, 256)).astype(np.int32)
    dg = orc.counts_to_delta(counts, f)
    for j in range(3):
        assert abs(np.sum(f * dg[j])) < 1e-10
        assert np.all(dg[j][f == 0] == 0)
    dg1 = orc.counts_to_delta(counts, None)
    for j in range(3):
        nhat = counts[j].mean()
        assert np.allclose(dg1[j], counts[j] / nhat - 1, rtol=1e-13, atol=1e-13)
    assert np.all(orc.counts_to_delta(np.zeros((1, 8), np.int32)) == 0)


def test_mean_cov_matches_numpy(orc):
    pk = np.random.default_rng(6).random((37, 5))
    mean, cov = orc.mean_cov(pk)
    assert np.allclose(mean, pk.mean(0), rtol=1e-14)
    assert np.allclose(cov, np.cov(pk, rowvar=False), rtol=1e-12)


def test_bin_edges(orc):
    lin = orc.bin_edges(orc.BINS_LINEAR, 64, 0.0, 256.0)
    assert np.array_equal(lin, np.arange(65) * 4.0)
    lg = orc.bin_edges(orc.BINS_LOG, 20, 1.0, 64.0)
    assert np.allclose(lg, np.geomspace(1.0, 64.0, 21), rtol=1e-14)
    ex = orc.bin_edges(orc.BINS_EDGES, 3, 0, 0, edges=[0.5, 1.0, 3.0, 7.0])
    assert list(ex) == [0.5, 1.0, 3.0, 7.0]
