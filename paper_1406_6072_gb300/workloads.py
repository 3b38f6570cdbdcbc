"""Synthetic workloads and seeded input generators.

This module holds no arithmetic of the method: only the sizes, correlation
parameters, seeds and realization counts of the workloads, plus seeded
generators of auxiliary inputs (survey masks, tabulated correlation rows,
serving request streams).  Both the CUDA path's tests/benchmark and the
oracle draw their inputs from here.

Correlation families (xi as a function of the physical lag r):
  gaussian       amp * exp(-r^2 / (2 scale^2))
  gen_cauchy     amp / (1 + (r/scale)^2)^beta
  exponential    amp * exp(-r / scale)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

XI_GAUSSIAN, XI_GEN_CAUCHY, XI_EXPONENTIAL, XI_TABLE = 0, 1, 2, 3


@dataclass(frozen=True)
class Workload:
    name: str
    n: tuple                 # survey cells per axis; the periodic grid is 2n per axis
    xi_kind: int
    amp: float
    scale: float
    beta: float
    dtype: str               # "f64" or "f32" per-realization arithmetic
    R: int                   # realizations (each gives two fields, Re and Im)
    seed: int
    clamp: bool              # clamp negative eigenvalues (family not PSD on 2n)
    sigma2: float | None = None   # variance of G used by the lognormal transform
    nbar: float | None = None     # Poisson intensity per cell with f = 1
    nbins: int | None = None      # power-spectrum bins, linear in |n| over [0, n/2)
    cell: tuple = field(default=(1.0, 1.0, 1.0))
    text: str = ""
    factor: int = 2                 # embedded side / survey side

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def m(self) -> tuple:
        return tuple(self.factor * v for v in self.n)

    @property
    def cells_per_field(self) -> int:
        return int(np.prod(self.n))

    @property
    def fields(self) -> int:
        return 2 * self.R


CONFIGS = {
    "gauss2d_n64_f64": Workload(
        "gauss2d_n64_f64", (64, 64), XI_GAUSSIAN, 1.0, 4.0, 0.0, "f64", 16, 1, False,
        text="2D 64x64 survey in a 128x128 periodic grid, xi = exp(-r^2/32), binary64, "
             "16 realizations (32 fields), seed 1"),
    "cauchy2d_n512_f32": Workload(
        "cauchy2d_n512_f32", (512, 512), XI_GEN_CAUCHY, 0.8, 8.0, 0.4, "f32", 64, 2, True,
        sigma2=0.8, nbar=2.0, nbins=64,
        text="2D 512x512 survey in 1024x1024, xi = 0.8/(1+(r/8)^2)^0.4 (clamped), binary32 "
             "fields with binary64 eigenvalues, 64 realizations, lognormal + Poisson nbar=2, "
             "64-bin power spectrum with mean and covariance, seed 2"),
    "exp3d_n128": Workload(
        "exp3d_n128", (128, 128, 128), XI_EXPONENTIAL, 1.0, 6.0, 0.0, "f32", 8, 3, False,
        sigma2=1.0, nbar=0.5, nbins=48,
        text="3D 128^3 survey in 256^3, xi = exp(-r/6), binary32, batch of 8 realizations, "
             "lognormal + Poisson nbar=0.5, 48 spherical shells, seed 3"),
    "mock_n128": Workload(
        "mock_n128", (128, 128), XI_GEN_CAUCHY, 0.14, 4.0, 0.4, "f32", 2000, 6, True,
        sigma2=float(np.log1p(0.14)), nbar=9.68, nbins=20,
        text="2D 128^2 survey in 256^2 (the paper's map size), density correlation "
             "omega = 0.14/(1+(r/4)^2)^0.4 embedded as ln(1+omega), lognormal sigma_A^2 = ln 1.14, "
             "Poisson nbar = 9.68 with a survey mask, 20 log-spaced bins, 2000 realizations, seed 6"),
    "cauchy2d_n2048_sweep": Workload(
        "cauchy2d_n2048_sweep", (2048, 2048), XI_GEN_CAUCHY, 0.8, 16.0, 0.4, "f32", 32, 4, True,
        nbins=64,
        text="2D 2048^2 survey in 4096^2, xi = 0.8/(1+(r/16)^2)^0.4 (clamped), 32 realizations, "
             "precision sweep, seed 4"),
    "cauchy2d_n512_padding": Workload(
        "cauchy2d_n512_padding", (512, 512), XI_GEN_CAUCHY, 0.8, 8.0, 0.4, "f32", 64, 2, True,
        sigma2=0.8, nbar=2.0, nbins=64,
        text="the 2D 512^2 workload embedded in 1024^2, 2048^2 and 4096^2 (factors 2, 4, 8): clamping "
             "error against cost, 64 realizations, lognormal + Poisson, 64-bin spectra, seed 2"),
    "exp3d_n256_sweep": Workload(
        "exp3d_n256_sweep", (256, 256, 256), XI_EXPONENTIAL, 1.0, 8.0, 0.0, "f32", 4, 8, False,
        nbins=64,
        text="3D 256^3 survey in 512^3, xi = exp(-r/8), 4 realizations, precision sweep, seed 8"),
}


def survey_mask(n, seed, masked_fraction=0.1, partial_fraction=0.2):
    """Seeded surface-fraction map f in [0,1] with fully masked (0), partial
    (0.7..1) and clean (1) cells, shaped like a survey mask."""
    rng = np.random.default_rng(seed)
    f = np.ones(tuple(n), dtype=np.float32)
    u = rng.random(tuple(n))
    f[u < partial_fraction] = rng.uniform(0.7, 1.0, size=int((u < partial_fraction).sum()))
    f[u < masked_fraction] = 0.0
    return f


def gaussian_field_values(shape, seed, scale=1.0):
    """Seeded standard-normal values (used as stand-in Gaussian fields)."""
    return (np.random.default_rng(seed).standard_normal(shape) * scale)


def serving_requests(count, seed=5, rate_hz=1000.0):
    """Seeded request stream of the mixed serving workload: Poisson arrivals,
    2D sides {64..1024} or 3D sides {32..128}, family gaussian or gen_cauchy
    (beta 0.4), amplitude U(0.2, 1.5), scale from {2,4,6,8,12,16}, 1..32
    realizations."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for i in range(count):
        if rng.random() < 0.5:
            side = int(rng.choice([64, 128, 256, 512, 1024]))
            n = (side, side)
        else:
            side = int(rng.choice([32, 64, 128]))
            n = (side, side, side)
        kind = XI_GAUSSIAN if rng.random() < 0.5 else XI_GEN_CAUCHY
        out.append({
            "id": i, "t_arrival": float(t[i]), "n": n, "xi_kind": kind,
            "amp": float(rng.uniform(0.2, 1.5)), "scale": float(rng.choice([2, 4, 6, 8, 12, 16])),
            "beta": 0.4 if kind == XI_GEN_CAUCHY else 0.0,
            "R": int(rng.integers(1, 33)), "seed": int(rng.integers(0, 2**62)),
        })
    return out
