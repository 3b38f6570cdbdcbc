"""The paper's printed parameter values as a worked example (CPU only).

Eq. (Lncov) at zero lag gives sigma_A^2 = ln(1 + sigma_delta^2); the paper
prints sigma_delta^2 = 0.14 and sigma_A^2 ~ 0.13.  The oracle's lognormal
step, fed a Gaussian with that variance and mean -sigma_A^2/2, must give
density fluctuations with variance 0.14 and Poisson counts with mean nbar.
"""
import json
import math
import os

import numpy as np

from paper_1406_6072_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def test_lncov_zero_lag_reproduces_printed_sigma2_A():
    s2d = GOLD["sigma2_delta"]["value"]
    assert round(math.log(1 + s2d), GOLD["sigma2_A"]["digits"]) == GOLD["sigma2_A"]["value"]


def test_embedding_is_twice_the_survey():
    assert GOLD["embedding_cells_per_side"]["value"] == 2 * GOLD["survey_cells_per_side"]["value"]


def test_lognormal_poisson_with_paper_values(orc):
    s2d = GOLD["sigma2_delta"]["value"]
    nbar = GOLD["nbar"]["value"]
    s2a = math.log(1 + s2d)
    n = GOLD["survey_cells_per_side"]["value"]
    G = W.gaussian_field_values((16, n * n), seed=21, scale=math.sqrt(s2a))
    delta, counts, _ = orc.lognormal_poisson(G, s2a, nbar, seed=22)
    assert abs(delta.var() / s2d - 1) < 0.03
    assert abs(counts.mean() / nbar - 1) < 0.01
    # practically all counts fall in the printed histogram range 0..41
    assert np.mean(counts <= GOLD["cic_N_max"]["value"]) > 0.9999
