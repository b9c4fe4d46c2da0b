"""Pins of the FP64 torch restatement used for reference gradients.

- Its forward equals the C oracle (Algorithm 1) after K iterations.
- Its autograd gradients of L = ||X_K - X_true||^2 with respect to mu_s,
  mu_nu, the tied rho and y (along a random unit direction) equal central
  finite differences of the C oracle.  The step (1e-7) is small enough that
  no threshold decision flips between the +h and -h runs in any iteration
  (at 1e-6 one coefficient of this cube crosses mu_s/rho and the difference
  quotient straddles the kink).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import torch_ref  # noqa: E402
from paper_1504_06847_gb300 import synth  # noqa: E402

K = 6
J = 2
BASE = dict(mu_eps=0.001, mu_s=0.05, mu_nu=0.01, rho=1.0)


def _params(mu_s, mu_nu, rho):
    return dict(mu_eps=BASE["mu_eps"], mu_s=mu_s, mu_nu=mu_nu, rho_P=rho, rho_T=rho, rho_V=rho, rho_S=rho)


def _oracle_loss(c, mu_s, mu_nu, rho, y=None):
    pb = oracle.Problem(c.psf, c.y if y is None else y, _params(mu_s, mu_nu, rho), J=J)
    st, _ = pb.run(K)
    return float(((st["X"] - c.sky) ** 2).sum()), st


@pytest.fixture(scope="module")
def cube():
    return synth.make_cube(32, 4, n_sources=3, n_antennas=24, seed=17)


@pytest.fixture(scope="module")
def ref(cube):
    return torch_ref.loss_and_grads(cube.psf, cube.y, cube.sky, BASE["mu_s"], BASE["mu_nu"], BASE["rho"], K, J=J)


def test_forward_equals_c_oracle(cube, ref):
    loss_c, st = _oracle_loss(cube, BASE["mu_s"], BASE["mu_nu"], BASE["rho"])
    assert np.max(np.abs(ref[5] - st["X"])) < 1e-12
    assert abs(ref[0] - loss_c) < 1e-10 * max(loss_c, 1.0)


@pytest.mark.parametrize("which", ["mu_s", "mu_nu", "rho"])
def test_scalar_gradients_match_finite_differences(cube, ref, which):
    h = 1e-7
    p = dict(mu_s=BASE["mu_s"], mu_nu=BASE["mu_nu"], rho=BASE["rho"])
    pp, pm = dict(p), dict(p)
    pp[which] += h
    pm[which] -= h
    lp, sp = _oracle_loss(cube, **pp)
    lm, sm = _oracle_loss(cube, **pm)
    # no threshold decision may flip between the two runs
    for key in ("P", "T", "V"):
        assert np.array_equal(sp[key] != 0, sm[key] != 0), key
    fd = (lp - lm) / (2 * h)
    g = {"mu_s": ref[2], "mu_nu": ref[3], "rho": ref[4]}[which]
    assert abs(g - fd) <= 1e-6 * max(abs(fd), 1.0), (which, g, fd)


def test_y_gradient_directional(cube, ref):
    rng = np.random.default_rng(3)
    d = rng.normal(size=cube.y.shape)
    d /= np.linalg.norm(d)
    h = 1e-7
    lp, sp = _oracle_loss(cube, BASE["mu_s"], BASE["mu_nu"], BASE["rho"], y=cube.y + h * d)
    lm, sm = _oracle_loss(cube, BASE["mu_s"], BASE["mu_nu"], BASE["rho"], y=cube.y - h * d)
    for key in ("P", "T", "V"):
        assert np.array_equal(sp[key] != 0, sm[key] != 0), key
    fd = (lp - lm) / (2 * h)
    g = float(np.sum(ref[1] * d))
    assert abs(g - fd) <= 1e-6 * max(abs(fd), 1.0), (g, fd)
