"""Pins of the oracle's spectral-index fit (the post-processing of the paper's
first simulation, Section 4: each pixel spectrum fitted in a log scale by the
second-order power law log S = c + alpha log(nu/nu0) + beta log^2(nu/nu0)).

- Spectra that are exactly of that form, with the curvature of the synthetic
  recipe, give back their own (log S0, alpha, beta).
- On the paper's two-Gaussian sky (constant spectral indices -1 and +1), the
  fit at each profile's centre gives its index up to the small admixture of
  the other profile, and a pixel with a non-positive value has no fit.
"""

import numpy as np

import oracle
from paper_1504_06847_gb300 import synth


def test_exact_curved_power_laws_are_recovered():
    rng = np.random.default_rng(7)
    nu = 1.025 + 0.05 * np.arange(15)
    N = 8
    s0 = rng.uniform(0.1, 2.0, size=(N, N))
    al = rng.uniform(-1.0, 0.5, size=(N, N))
    be = rng.uniform(-0.2, 0.2, size=(N, N))
    u = np.log(nu / nu[0])[:, None, None]
    cube = s0 * np.exp((al + be * u) * u)
    c, a, b = oracle.spectral_index(cube, nu)
    assert np.max(np.abs(c - np.log(s0))) < 1e-12
    assert np.max(np.abs(a - al)) < 1e-11
    assert np.max(np.abs(b - be)) < 1e-10


def test_two_gaussian_sky_indices():
    sigma = 3.0
    g = synth.two_gaussians(N=64, L=15, sigma_px=sigma)
    c, a, b = oracle.spectral_index(g.sky, g.nu)
    row = 32
    # at one centre the other profile adds eps (nu/nu0)^(+-1), eps = exp(-d^2 / (2 sigma^2)),
    # which moves the fitted slope by about 2 eps (log(1 + eps x^2) ~ eps (1 + 2 log x))
    eps = np.exp(-(37 - 27) ** 2 / (2 * sigma ** 2))
    assert abs(a[row, 27] + 1.0) < 3 * eps  # centre of the alpha = -1 profile (pixel 108 of 256)
    assert abs(a[row, 37] - 1.0) < 3 * eps  # centre of the alpha = +1 profile (pixel 148 of 256)
    assert abs(a[row, 27] + 1.0) > 0.5 * eps  # the admixture is there, and of the predicted size
    cube = g.sky.copy()
    cube[3, 0, 0] = 0.0
    _, a2, _ = oracle.spectral_index(cube, g.nu, floor=0.0)
    assert np.isnan(a2[0, 0]) and np.isfinite(a2[row, 27])
