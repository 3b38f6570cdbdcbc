"""The binary32 Poisson walk's acceptance bound (section 3.1, eq. (sampling)).

The sampler decides each count n = min{j : U < F(j; mu)} with a binary32 walk
and hands it to the binary64 walk whenever U lies within a bound on the
binary32 error of one of the two CDF values that decide it.  This test models
that fast path in numpy binary32 arithmetic, with every library exponential
and quotient pushed to the edge of its documented error (2 ulp) in a random
direction, and places U adversarially close to the CDF values: every count
the model accepts must equal the exact decision.  The same model with a bound
fifty times smaller must accept wrong counts, which shows the cases reach the
band's edge.  A last test runs the binary64 walk that decides the remaining
counts with its term tests in floating point and in the integer form the
kernel uses (j > floor(mu), U < F and F + p == F on the bit patterns): the
same counts.
"""
import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")

F32 = np.float32
U_RND = 2.0 ** -24


def _edge(x, rng):
    """x (binary32) moved by up to 2 ulp in a random direction."""
    s = rng.choice(np.array([-1.0, 1.0]), size=x.shape)
    return (x.astype(np.float64) * (1.0 + s * 4.0 * U_RND * rng.random(x.shape))).astype(F32)


def _fast_path(G, hs, nbar, f, ubits, rng, tol_scale=1.0):
    """The binary32 walk and its acceptance test; -1 where binary64 decides."""
    G = G.astype(F32)
    hs_f, nbar_f = F32(hs), F32(nbar)
    mu = (nbar_f * f.astype(F32)) * _edge(np.exp(G - hs_f), rng)
    Uf = ((ubits >> np.uint64(30)).astype(np.float64) * 2.0 ** -23).astype(F32)
    p0 = _edge(np.exp(-mu), rng)
    p1 = p0 * mu
    p2 = p1 * (mu * F32(0.5))
    p3 = p2 * (mu * F32(1.0 / 3.0))
    F0 = p0
    F1 = F0 + p1
    F2 = F1 + p2
    F3 = F2 + p3
    zero = np.zeros_like(F0)
    j = np.where(Uf < F0, 0, np.where(Uf < F1, 1, np.where(Uf < F2, 2, 3)))
    F = np.where(Uf < F0, F0, np.where(Uf < F1, F1, np.where(Uf < F2, F2, F3)))
    Fp = np.where(Uf < F0, zero, np.where(Uf < F1, F0, np.where(Uf < F2, F1, F2)))
    p = p3.copy()
    walking = ~(Uf < F3)
    while np.any(walking & (j < 400)):
        w = walking & ~(Uf < F) & (j < 400)
        if not np.any(w):
            break
        j = np.where(w, j + 1, j)
        p = np.where(w, p * _edge(mu / np.maximum(j, 1).astype(F32), rng), p)
        Fp = np.where(w, F, Fp)
        F = np.where(w, F + p, F)
    fj = j.astype(F32)
    tol = F32(1.2e-7 * tol_scale) * (F32(6) + F32(6) * fj + (F32(7) + np.abs(G) + F32(2) * hs_f) * mu)
    ok = (mu < 80) & (mu > 0) & (j < 400) & ((F - Uf) > tol) & ((j == 0) | ((Uf - Fp) > tol))
    return np.where(ok, j, -1)


def _cases(rng, n, sigma2, nbar):
    """Cells whose U sits within a few bounds of a CDF value of their count."""
    G = rng.normal(0.0, np.sqrt(sigma2), n)
    G[: n // 20] *= 3.0  # the tails of G
    G = G.astype(F32).astype(np.float64)
    f = np.where(rng.random(n) < 0.5, 1.0, rng.random(n)).astype(F32).astype(np.float64)
    mu = nbar * f * np.exp(G - 0.5 * sigma2)
    keep = (mu > 1e-6) & (mu < 79.0)
    G, f, mu = G[keep], f[keep], mu[keep]
    jstar = scipy_stats.poisson.ppf(rng.random(len(mu)), mu).astype(np.int64)
    Fj = scipy_stats.poisson.cdf(jstar, mu)
    band = 1.2e-7 * (6 + 6 * (jstar + 1) + (7 + np.abs(G) + sigma2) * mu)
    delta = rng.uniform(-2.0, 2.0, len(mu)) * band
    delta = np.where(np.abs(delta) < 1e-12, 1e-12, delta)
    U = np.clip(Fj + delta, 0.0, 1.0 - 2.0 ** -53)
    ubits = np.floor(U * 2.0 ** 53).astype(np.uint64)
    U = ubits.astype(np.float64) * 2.0 ** -53
    # exact decision: U < F(jstar) gives jstar, otherwise jstar + 1, as long
    # as U stays between the neighbouring CDF values (cases where a term is
    # smaller than the offset are dropped)
    jtrue = np.where(U < Fj, jstar, jstar + 1)
    lo = np.where(jtrue > 0, scipy_stats.poisson.cdf(jtrue - 1, mu), -1.0)
    hi = scipy_stats.poisson.cdf(jtrue, mu)
    good = (lo <= U) & (U < hi)
    assert np.count_nonzero(good) > len(U) // 2
    return G[good], f[good], ubits[good], jtrue[good]


@pytest.mark.parametrize("sigma2,nbar", [(0.8, 2.0), (0.1, 30.0), (3.0, 0.05), (0.8, 0.5)])
def test_accepted_binary32_counts_are_exact(sigma2, nbar):
    rng = np.random.default_rng(int(sigma2 * 1000 + nbar * 10))
    G, f, ubits, jtrue = _cases(rng, 200_000, sigma2, nbar)
    j = _fast_path(G, 0.5 * sigma2, nbar, f, ubits, rng)
    acc = j >= 0
    assert np.count_nonzero(acc) > len(j) // 4
    assert np.array_equal(j[acc], jtrue[acc])


def test_a_smaller_bound_accepts_wrong_counts():
    rng = np.random.default_rng(7)
    G, f, ubits, jtrue = _cases(rng, 200_000, 0.8, 2.0)
    j = _fast_path(G, 0.4, 2.0, f, ubits, rng, tol_scale=1.0 / 50.0)
    acc = j >= 0
    assert np.count_nonzero(j[acc] != jtrue[acc]) > 0


def _walk_float_tests(U, mu, inv):
    """The binary64 walk with its tests in floating point (j > mu, U < F,
    F + p == F)."""
    j, p = 0, np.exp(-mu)
    F = p
    while not (U < F):
        j += 1
        p = p * (mu * inv[j])
        Fn = F + p
        if Fn == F and float(j) > mu:
            break
        F = Fn
    return j


def _walk_integer_tests(U, mu, inv):
    """The same walk with the tests the kernel makes in integers: j > floor(mu)
    and the comparisons on the doubles' bit patterns."""
    bits = lambda x: int(np.float64(x).view(np.int64))
    jm, Ub = int(np.floor(mu)), bits(U)
    j, p = 0, np.exp(-mu)
    F = p
    while not (Ub < bits(F)):
        j += 1
        p = p * (mu * inv[j])
        Fn = F + p
        if j > jm and bits(Fn) == bits(F):
            break
        F = Fn
    return j


def test_walk_integer_tests_match_float_tests():
    rng = np.random.default_rng(5)
    inv = np.array([0.0] + [1.0 / i for i in range(1, 2048)])
    mus = np.concatenate([rng.uniform(0.01, 30.0, 300), rng.uniform(30.0, 700.0, 60),
                          np.arange(1.0, 40.0), [700.0, 699.5, 1e-3]])
    for mu in mus:
        for U in (rng.random(), 0.0, 1.0 - 2.0 ** -53, rng.random() ** 8, 1.0 - rng.random() ** 8):
            assert _walk_integer_tests(U, float(mu), inv) == _walk_float_tests(U, float(mu), inv)
