"""Pins for the oracle's random-number side (CPU only).

The paper only asks for independent zero-mean Gaussian modes (section 2,
eq. (Papos2)); the generator is this project's specification.  These tests pin
the oracle's implementation of that specification against things other than
itself:
  * Philox4x32-10 against Triton's independent implementation (CPU interpreter);
  * the own ln / cos / sin against numpy and mpmath;
  * the bit layout of the uniforms against Triton's words + numpy's math;
  * the distribution of the noise (KS normality, moments, independence).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_words(requests):
    pytest.importorskip("triton")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")],
                          input=json.dumps(requests), capture_output=True, text=True,
                          timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    return [np.asarray(r, dtype=np.uint64).astype(np.uint32) for r in json.loads(proc.stdout)]


@pytest.fixture(scope="module")
def triton_cases():
    rng = np.random.default_rng(20140623)
    seeds = [0, 1, 2, 0xFFFFFFFF, 0x123456789ABCDEF0, int(rng.integers(0, 2**63))]
    reqs = []
    for s in seeds:
        ctrs = rng.integers(0, 2**32, size=(37, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = [2**32 - 1] * 4
        ctrs[2] = [5, 0, 3, 0]
        ctrs[3] = [5, 0, 3, 1]
        reqs.append([int(s), ctrs.tolist()])
    return reqs, _triton_words(reqs)


def test_philox_matches_independent_implementation(orc, triton_cases):
    reqs, words = triton_cases
    for (seed, ctrs), expect in zip(reqs, words):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for ctr, e in zip(ctrs, expect):
            got = orc.philox(ctr, key)
            assert np.array_equal(got, e), (seed, ctr, got, e)


def _ulps(a, b, dtype):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    sp = np.spacing(np.abs(b).astype(dtype)).astype(np.float64)
    return np.abs(a - b) / sp


def test_log_unit_accuracy(orc):
    import mpmath as mp
    rng = np.random.default_rng(1)
    ints = np.concatenate([np.arange(1, 2000), rng.integers(1, 2**53, 4000),
                           2**53 - np.arange(0, 2000), [2**52, 2**51 + 1]])
    u = (ints.astype(np.float64)) * 2.0**-53
    got = np.array([orc.log_unit(x) for x in u])
    ref = np.array([float(mp.log(mp.mpf(x))) for x in u])
    assert np.all(_ulps(got, ref, np.float64)[ref != 0] <= 2.0)
    assert orc.log_unit(1.0) == 0.0
    # binary32 version on the binary32 uniform lattice k 2^-24
    k = np.concatenate([np.arange(1, 3000), rng.integers(1, 2**24, 5000), 2**24 - np.arange(0, 3000)])
    uf = (k.astype(np.float32) * np.float32(2.0**-24)).astype(np.float32)
    gotf = np.array([orc.logf_unit(x) for x in uf], dtype=np.float32)
    reff = np.log(uf.astype(np.float64))
    assert np.all(_ulps(gotf, reff, np.float32)[reff != 0] <= 2.0)


def test_cossin_2pi_accuracy(orc):
    import mpmath as mp
    mp.mp.prec = 120
    rng = np.random.default_rng(2)
    ints = np.concatenate([np.arange(1, 600), rng.integers(1, 2**53, 3000),
                           [2**50, 2**51, 3 * 2**50, 2**53, 2**53 - 1, 2**50 + 1]])
    u = ints.astype(np.float64) * 2.0**-53
    for x in u:
        c, s = orc.cossin_2pi(x)
        cr = float(mp.cos(2 * mp.pi * mp.mpf(x)))
        sr = float(mp.sin(2 * mp.pi * mp.mpf(x)))
        assert abs(c - cr) <= 2.5e-16 and abs(s - sr) <= 2.5e-16, (x, c - cr, s - sr)
    k = np.concatenate([np.arange(1, 500), rng.integers(1, 2**24, 3000), [2**22, 2**23, 2**24]])
    uf = (k.astype(np.float32) * np.float32(2.0**-24)).astype(np.float32)
    for x in uf:
        c, s = orc.cossin_2pif(x)
        cr = np.cos(2 * np.pi * np.float64(x))
        sr = np.sin(2 * np.pi * np.float64(x))
        assert abs(c - cr) <= 1.5e-7 and abs(s - sr) <= 1.5e-7, (x, c - cr, s - sr)
    # exact quarter turns
    assert orc.cossin_2pi(1.0) == (1.0, 0.0)
    assert orc.cossin_2pi(0.25) == (0.0, 1.0)
    assert orc.cossin_2pi(0.5) == (-1.0, 0.0)


def _uniform53(a, b):
    return (((a.astype(np.uint64) >> np.uint64(5)) << np.uint64(26)) | (b.astype(np.uint64) >> np.uint64(6))).astype(np.float64)


def test_noise_bit_layout_against_independent_pieces(orc):
    """Noise = Box-Muller of uniforms built from Philox words; rebuilt here from
    Triton's Philox and numpy's log/cos/sin (agreement to rounding)."""
    seed, r, m_last = 0x0000000200000007, 3, 8
    ncells = 2 * m_last
    # binary64: one counter per cell (k_lo, k_hi, r, 0)
    reqs = [[seed, [[k, 0, r, 0] for k in range(ncells)]],
            [seed, [[p, 0, r, 0] for p in range(ncells // 2)]]]
    w64, w32 = _triton_words(reqs)
    eps = orc.draw_noise(seed, r, 1, ncells, m_last, 0)[0]
    u1 = (_uniform53(w64[:, 0], w64[:, 1]) + 1.0) * 2.0**-53
    u2 = (_uniform53(w64[:, 2], w64[:, 3]) + 1.0) * 2.0**-53
    rad = np.sqrt(-2.0 * np.log(u1))
    ref = rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)
    assert np.max(np.abs(eps - ref)) < 1e-13
    # binary32: pair p = row*(M/2) + (col mod M/2); lower half words 0,1; upper 2,3
    eps32 = orc.draw_noise(seed, r, 1, ncells, m_last, 1)[0]
    ref32 = np.zeros(ncells, dtype=np.complex128)
    for k in range(ncells):
        row, col = divmod(k, m_last)
        p = row * (m_last // 2) + col % (m_last // 2)
        a, b = (w32[p, 2], w32[p, 3]) if col >= m_last // 2 else (w32[p, 0], w32[p, 1])
        ua = ((int(a) >> 8) + 1) * 2.0**-24
        ub = ((int(b) >> 8) + 1) * 2.0**-24
        rr = np.sqrt(-2.0 * np.log(ua))
        ref32[k] = rr * np.cos(2 * np.pi * ub) + 1j * rr * np.sin(2 * np.pi * ub)
    assert np.max(np.abs(eps32 - ref32)) < 4e-6
    # the binary32 draws are exactly representable in binary32
    assert np.all(eps32.real.astype(np.float32).astype(np.float64) == eps32.real)


def test_poisson_uniform_layout(orc):
    seed = 77
    reqs = [[seed, [[c, 0, f >> 1, 1] for c in range(6) for f in range(4)]]]
    (w,) = _triton_words(reqs)
    i = 0
    for c in range(6):
        for f in range(4):
            a, b = (w[i, 2], w[i, 3]) if f & 1 else (w[i, 0], w[i, 1])
            ref = float(_uniform53(np.array([a]), np.array([b]))[0]) * 2.0**-53
            assert orc.poisson_uniform(seed, c, f) == ref
            i += 1


@pytest.mark.parametrize("dtype", [0, 1])
def test_noise_distribution(orc, dtype):
    from scipy import stats
    m_last = 64
    eps = orc.draw_noise(12345, 0, 4, 64 * m_last, m_last, dtype).ravel()
    x = np.concatenate([eps.real, eps.imag])
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(stats.kurtosis(x)) < 5 * np.sqrt(24 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # independence: Re/Im of a cell, neighbouring cells, paired columns, realizations
    e = eps.reshape(4, 64, m_last)
    lim = 5 / np.sqrt(e[..., :].size)
    assert abs(np.corrcoef(e.real.ravel(), e.imag.ravel())[0, 1]) < lim
    assert abs(np.corrcoef(e.real[..., :-1].ravel(), e.real[..., 1:].ravel())[0, 1]) < lim * 1.1
    h = m_last // 2
    assert abs(np.corrcoef(e.real[..., :h].ravel(), e.real[..., h:].ravel())[0, 1]) < lim * 1.5
    assert abs(np.corrcoef(e.real[0].ravel(), e.real[1].ravel())[0, 1]) < lim * 2
    # different seeds give different draws
    other = orc.draw_noise(12346, 0, 1, 64, m_last, dtype)
    assert not np.allclose(other[0], eps[:64])
