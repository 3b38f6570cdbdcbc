"""Plain FP64 CPU oracle of the exact circulant-embedding sampler (Carron,
Wolk & Szapudi 2014) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library and its Python
binding never import it; the two implementations share no code.

The arithmetic of the sampler lives in ``cf_oracle.c`` (plain C, binary64,
compiled with ``-ffp-contract=off``); this module builds/loads it and
marshals numpy arrays.  ``build()`` compiles it with gcc.  The counts-in-cells
functions of section 3.4 (histogram, mixture prediction, A*) are written here
in plain numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cf_oracle.c")
_LIB = os.path.join(_HERE, "_cf_oracle.so")
_lib = None

XI_GAUSSIAN, XI_GEN_CAUCHY, XI_EXPONENTIAL, XI_TABLE = 0, 1, 2, 3
BINS_LINEAR, BINS_LOG, BINS_EDGES = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``_cf_oracle.so`` (gcc, -O2, no FP contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "cf_oracle.h")))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Report(C.Structure):
    _fields_ = [("lambda_min", C.c_double), ("lambda_max", C.c_double), ("tau", C.c_double),
                ("neg_mass", C.c_double), ("cov_error", C.c_double),
                ("n_negative", C.c_int64), ("n_zeroed", C.c_int64),
                ("clamped", C.c_int32), ("status", C.c_int32)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p


def _lib_handle():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.or_philox4x32_10.argtypes = [_P, _P, _P]
        lib.or_log_unit.argtypes = [C.c_double]
        lib.or_log_unit.restype = C.c_double
        lib.or_logf_unit.argtypes = [C.c_float]
        lib.or_logf_unit.restype = C.c_float
        lib.or_cossin_2pi.argtypes = [C.c_double, _P, _P]
        lib.or_cossin_2pif.argtypes = [C.c_float, _P, _P]
        lib.or_draw_noise.argtypes = [C.c_uint64, C.c_uint64, C.c_int32, C.c_int64, C.c_int64,
                                      C.c_int32, _P]
        lib.or_dft_naive.argtypes = [_P, _P, C.c_int64, C.c_int]
        lib.or_fft_recursive.argtypes = [_P, C.c_int64, C.c_int]
        lib.or_fft_nd.argtypes = [_P, C.c_int32, _P, C.c_int]
        lib.or_embed_row.argtypes = [C.c_int32, _P, _P, C.c_int32, C.c_double, C.c_double,
                                     C.c_double, _P, _P]
        lib.or_eigenvalues.argtypes = [C.c_int32, _P, _P, _P]
        lib.or_psd.argtypes = [C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P, C.POINTER(Report)]
        lib.or_sample.argtypes = [C.c_int32, _P, _P, _P, C.c_uint64, C.c_uint64, C.c_int32,
                                  C.c_int32, _P]
        lib.or_sample_given_noise.argtypes = [C.c_int32, _P, _P, _P, _P, _P]
        lib.or_poisson_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        lib.or_poisson_uniform.restype = C.c_double
        lib.or_poisson_icdf.argtypes = [C.c_double, C.c_double, _P]
        lib.or_poisson_icdf.restype = C.c_int32
        lib.or_lognormal_poisson.argtypes = [_P, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                             _P, C.c_uint64, C.c_uint64, _P, _P, _P]
        lib.or_bin_edges.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, _P, _P]
        lib.or_power_spectrum.argtypes = [_P, C.c_int32, _P, _P, C.c_int64, C.c_int32,
                                          _P, _P, _P]
        lib.or_counts_to_delta.argtypes = [_P, _P, C.c_int64, C.c_int64, _P]
        lib.or_mean_cov.argtypes = [_P, C.c_int64, C.c_int32, _P, _P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dims(n):
    n = [int(v) for v in n]
    return np.asarray(n + [1] * (3 - len(n)), dtype=np.int64), len(n)


# ---------------------------------------------------------------- generator
def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key -> 4 uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib_handle().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def log_unit(u: float) -> float:
    return _lib_handle().or_log_unit(float(u))


def logf_unit(u) -> np.float32:
    return np.float32(_lib_handle().or_logf_unit(float(u)))


def cossin_2pi(u: float):
    c, s = C.c_double(), C.c_double()
    _lib_handle().or_cossin_2pi(float(u), C.byref(c), C.byref(s))
    return c.value, s.value


def cossin_2pif(u):
    c, s = C.c_float(), C.c_float()
    _lib_handle().or_cossin_2pif(float(u), C.byref(c), C.byref(s))
    return np.float32(c.value), np.float32(s.value)


def draw_noise(seed, r0, R, ncells, m_last, dtype):
    """Complex noise [R][ncells] (complex128; dtype 1 values are exact binary32)."""
    out = np.zeros((R, ncells, 2), dtype=np.float64)
    _lib_handle().or_draw_noise(seed, r0, R, ncells, m_last, dtype, _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


# ---------------------------------------------------------------- transforms
def dft_naive(x, sign):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.zeros_like(x)
    _lib_handle().or_dft_naive(_ptr(x), _ptr(out), x.size, sign)
    return out


def fft_recursive(x, sign):
    a = np.array(x, dtype=np.complex128, copy=True)
    _lib_handle().or_fft_recursive(_ptr(a), a.size, sign)
    return a


def fft_nd(x, sign):
    a = np.array(x, dtype=np.complex128, copy=True, order="C")
    dims = np.asarray(a.shape, dtype=np.int64)
    _lib_handle().or_fft_nd(_ptr(a), a.ndim, _ptr(dims), sign)
    return a


# ---------------------------------------------------------------- embedding
def embed_row(n, kind, amp=1.0, scale=1.0, beta=0.0, cell=None, table=None, log1p=False, factor=2, M=None):
    """First row c of the circulant (step a1, section 2 eq. (grid)) on the
    embedded grid of `factor` times the survey side per axis (2: the paper's
    box of twice the side; a larger box embeds the same way, section 2, Fig. 1:
    any survey-sized sub-box of it has the target covariance).  log1p: xi is
    the correlation function of the lognormal density and the Gaussian
    covariance is ln(1 + xi) (section 3.1, eq. (Lncov)).  M: explicit
    embedded sides (any M_i >= 2 n_i), instead of factor * n."""
    d = len(n)
    cellv = np.ones(3) if cell is None else np.asarray(list(cell) + [1.0] * (3 - len(cell)))
    M = [int(factor) * int(v) for v in n] if M is None else [int(v) for v in M]
    mdims, _ = _dims(M)
    c = np.zeros(int(np.prod(M)), dtype=np.float64)
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.float64).ravel()
    _lib_handle().or_embed_row(d, _ptr(mdims), _ptr(cellv), kind, amp, scale, beta, _ptr(tab),
                               _ptr(c))
    if log1p:
        c = np.log1p(c)
    return c.reshape(M)


def _mdims(n, a):
    """Embedded sides: the shape of the M^d array `a` (survey sizes n)."""
    a = np.asarray(a)
    shape = a.shape if a.ndim == len(n) else (tuple(2 * int(v) for v in n) if a.ndim == 1 else a.shape)
    if int(np.prod(shape)) != a.size or len(shape) != len(n):
        raise ValueError("array does not have the embedded grid's shape")
    return _dims(shape)[0]


def eigenvalues(n, c):
    d = len(n)
    c = np.ascontiguousarray(c, dtype=np.float64)
    lam = np.zeros(c.size, dtype=np.float64)
    _lib_handle().or_eigenvalues(d, _ptr(_mdims(n, c)), _ptr(c), _ptr(lam))
    return lam.reshape(c.shape)


def psd(n, c, lam, clamp=False):
    dims, d = _dims(n)
    c = np.ascontiguousarray(c, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    lp = np.zeros_like(lam)
    s = np.zeros_like(lam)
    rep = Report()
    _lib_handle().or_psd(d, _ptr(dims), _ptr(_mdims(n, c)), _ptr(c), _ptr(lam), int(bool(clamp)), _ptr(lp),
                         _ptr(s), C.byref(rep))
    return lp, s, rep.asdict()


def embed(n, kind, amp=1.0, scale=1.0, beta=0.0, cell=None, table=None, clamp=False, log1p=False, factor=2,
          M=None):
    """Steps a1-a3: first row c, eigenvalues lambda, lambda+, sqrt(lambda+), report."""
    c = embed_row(n, kind, amp, scale, beta, cell, table, log1p, factor, M)
    lam = eigenvalues(n, c)
    lp, s, rep = psd(n, c, lam, clamp)
    return {"c": c, "lambda": lam, "lambda_plus": lp, "sqrt_lambda": s, "report": rep}


# ---------------------------------------------------------------- sampling
def sample(n, s, seed, r0, R, dtype):
    """Fields [R][2][*n] (Re, Im) from sqrt(lambda+) s; dtype 0 f64 noise, 1 f32 noise."""
    dims, d = _dims(n)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros((R, 2) + tuple(int(v) for v in n), dtype=np.float64)
    _lib_handle().or_sample(d, _ptr(dims), _ptr(_mdims(n, s)), _ptr(s), seed, r0, R, dtype, _ptr(out))
    return out


def sample_given_noise(n, s, eps):
    dims, d = _dims(n)
    s = np.ascontiguousarray(s, dtype=np.float64)
    e = np.ascontiguousarray(np.stack([np.real(eps), np.imag(eps)], axis=-1), dtype=np.float64)
    w = np.zeros(tuple(int(v) for v in n) + (2,), dtype=np.float64)
    _lib_handle().or_sample_given_noise(d, _ptr(dims), _ptr(_mdims(n, s)), _ptr(s), _ptr(e), _ptr(w))
    return w[..., 0] + 1j * w[..., 1]


# ---------------------------------------------------------------- lognormal / Poisson
def poisson_uniform(seed, cell, field):
    return _lib_handle().or_poisson_uniform(seed, cell, field)


def poisson_icdf(U, mu):
    m = C.c_double()
    n = _lib_handle().or_poisson_icdf(float(U), float(mu), C.byref(m))
    return n, m.value


def lognormal_poisson(G, sigma2, nbar, f=None, seed=0, field0=0):
    """G: [nfields][cells] -> (delta, counts int32, margin)."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    nf, cells = G.shape[0], int(np.prod(G.shape[1:]))
    fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64).ravel()
    delta = np.zeros_like(G)
    counts = np.zeros(G.shape, dtype=np.int32)
    margin = np.zeros_like(G)
    _lib_handle().or_lognormal_poisson(_ptr(G), cells, nf, sigma2, nbar, _ptr(fa), seed, field0,
                                       _ptr(delta), _ptr(counts), _ptr(margin))
    return delta, counts, margin


# ---------------------------------------------------------------- power spectrum
def bin_edges(kind, nbins, kmin, kmax, edges=None):
    e_in = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros(nbins + 1, dtype=np.float64)
    _lib_handle().or_bin_edges(kind, nbins, kmin, kmax, _ptr(e_in), _ptr(out))
    return out


def power_spectrum(fields, n, edges, cell=1.0):
    """Binned power spectrum, section 3.2 eq. (Def spec): fields [F][*n] ->
    (pk [F][nbins], nmodes [nbins]).  cell: one size for every axis or one
    per axis.  |k| is in units of the fundamental frequency of the longest
    side (the integer index length on a cube)."""
    dims, d = _dims(n)
    cellv = np.ones(3, dtype=np.float64)
    cellv[:d] = np.broadcast_to(np.asarray(cell, dtype=np.float64), (d,))
    fl = np.ascontiguousarray(fields, dtype=np.float64)
    F = fl.shape[0]
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nb = edges.size - 1
    pk = np.zeros((F, nb), dtype=np.float64)
    nm = np.zeros(nb, dtype=np.int64)
    _lib_handle().or_power_spectrum(_ptr(fl), d, _ptr(dims), _ptr(cellv), F, nb, _ptr(edges), _ptr(pk),
                                    _ptr(nm))
    return pk, nm


def counts_to_delta(counts, f=None):
    N = np.ascontiguousarray(counts, dtype=np.int32)
    nf, cells = N.shape[0], int(np.prod(N.shape[1:]))
    fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64).ravel()
    out = np.zeros(N.shape, dtype=np.float64)
    _lib_handle().or_counts_to_delta(_ptr(N), _ptr(fa), cells, nf, _ptr(out))
    return out


def mean_cov(pk):
    pk = np.ascontiguousarray(pk, dtype=np.float64)
    F, nb = pk.shape
    mean = np.zeros(nb)
    cov = np.zeros((nb, nb))
    _lib_handle().or_mean_cov(_ptr(pk), F, nb, _ptr(mean), _ptr(cov))
    return mean, cov


# ---------------------------------------------------------------- counts in cells (section 3.4)
def cic_histogram(counts, f, nbins):
    """P(N) = #{i : f_i != 0, N_i = N}, N < nbins, per map (rows of counts)."""
    counts = np.asarray(counts).reshape(len(counts), -1)
    keep = np.ones(counts.shape[1], bool) if f is None else (np.asarray(f).ravel() != 0)
    out = np.zeros((counts.shape[0], nbins), dtype=np.float64)
    for r, c in enumerate(counts):
        v = c[keep]
        v = v[(v >= 0) & (v < nbins)]
        out[r] = np.bincount(v, minlength=nbins)[:nbins]
    return out


def cic_prediction(sigma2, nbar, f, nbins):
    """<P(N)> = int dA N(A; -s^2/2, s^2) e^{NA}/N! sum_{f_i != 0} (nbar f_i)^N
    e^{-nbar f_i e^A} (section 3.4), for N < nbins, each N by adaptive
    quadrature (scipy.integrate.quad) over A in -s^2/2 +- 14 s, with a break
    point at the peak of the Poisson factor, A = ln((N + 1/2) / mean(nbar f))."""
    import math

    from scipy import integrate
    nb = nbar * (np.ones(1) if f is None else np.asarray(f, dtype=np.float64).ravel())
    nb = nb[nb > 0]
    lnb = np.log(nb)
    sd = math.sqrt(sigma2)
    lo, hi = -sigma2 / 2 - 14 * sd, -sigma2 / 2 + 14 * sd
    out = np.zeros(nbins)
    for N in range(nbins):
        lg = math.lgamma(N + 1)

        def integrand(A):
            gauss = math.exp(-(A + sigma2 / 2) ** 2 / (2 * sigma2)) / math.sqrt(2 * math.pi * sigma2)
            return gauss * float(np.sum(np.exp(N * (A + lnb) - nb * math.exp(A) - lg)))

        peak = min(max(math.log((N + 0.5) / nb.mean()), lo + 1e-9), hi - 1e-9)
        out[N] = integrate.quad(integrand, lo, hi, points=[peak], limit=400, epsabs=0.0, epsrel=1e-12)[0]
    return out


def astar(counts, f, nbar, sigma2):
    """A*(N) of eq. (As): the root of e^A nbar f_i s^2 + A = s^2 (N - 1/2), by
    bisection (the left side increases with A); 0 where f_i = 0."""
    counts = np.asarray(counts, dtype=np.float64)
    fb = np.ones(counts.shape[-1]) if f is None else np.asarray(f, dtype=np.float64).ravel()
    k = nbar * fb * sigma2
    c = sigma2 * (counts - 0.5)
    hi = c.copy()                        # e^A k >= 0, so the root is <= c
    lo = c - 60.0 - np.abs(c)            # k e^lo + lo - c < 0 there
    kk = np.broadcast_to(k, counts.shape)
    mask = kk > 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        g = kk * np.exp(mid) + mid - c
        lo = np.where(g < 0, mid, lo)
        hi = np.where(g < 0, hi, mid)
    return np.where(mask, 0.5 * (lo + hi), 0.0)


# ---------------------------------------------------------------- cumulative information (section 3.3)
def cumulative_information(mean, cov):
    """I(<= b) = sum_{b1, b2 <= b} [C_b^{-1}]_{b1 b2}, C_{12} = cov_{12} / (mean_1 mean_2)
    over the bins up to b with a positive mean (eq. (cuminfo)); bins without
    modes repeat the previous value.  Each prefix matrix is inverted directly."""
    mean = np.asarray(mean, dtype=np.float64)
    cov = np.asarray(cov, dtype=np.float64)
    keep = np.flatnonzero(mean > 0)
    out = np.zeros(len(mean))
    run = 0.0
    for b in range(len(mean)):
        sel = keep[keep <= b]
        if len(sel) and sel[-1] == b:
            Cb = cov[np.ix_(sel, sel)] / np.outer(mean[sel], mean[sel])
            run = float(np.sum(np.linalg.inv(Cb)))
        out[b] = run
    return out


# ---------------------------------------------------------------- periodic box (section 3.3)
def periodic_lambda(n, kind, amp, scale, beta, box_factor, extent, resolution, log1p=False):
    """Eigenvalues of the k-space sampler of eq. (Periodicboxmodes) on the
    sampler's embedding grid (2n per axis, or 4n for box_factor 4): a box of
    side B = box_factor n with modes k = 2 pi m / B of variance P(k) (cell 1),
    P the Fourier sum of xi on a grid of spacing 1/resolution and extent
    extent B, the DC mode zero; for box_factor 1 the modes sit on the even
    frequencies of the 2n grid with weight 2^d."""
    d = len(n)
    nb = [resolution * extent * box_factor * v // 2 for v in n]
    c = embed_row(nb, kind, amp, scale, beta, cell=[1.0 / resolution] * d, log1p=log1p)
    lam_big = eigenvalues(nb, c)
    Mb = lam_big.shape
    ne = [2 * v if box_factor == 4 else v for v in n]
    Me = [2 * v for v in ne]
    idx = np.indices(Me)
    zero = np.zeros(Me, dtype=bool)
    dc = np.ones(Me, dtype=bool)
    big_index = []
    for a in range(d):
        m = idx[a]
        if box_factor == 1:
            zero |= (m % 2) == 1
            m = m // 2
            B = Me[a] // 2
        else:
            B = Me[a]
        f = np.where(m < B // 2, m, m - B)
        dc &= f == 0
        big_index.append((extent * f) % Mb[a])
    scale_ = (1.0 / resolution) ** d * (2.0 ** d if box_factor == 1 else 1.0)
    lam = lam_big[tuple(big_index)] * scale_
    lam[zero | dc] = 0.0
    return lam
