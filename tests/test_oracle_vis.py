"""Pins of the oracle's visibility-domain operator (Section 2, last paragraph:
y_l are the sampled visibilities and H_l maps the sky to them) and of step I
solved for it by conjugate gradients.

- At integer uv coordinates the operator is the 2-D DFT that numpy's FFT
  computes, up to the phase (-1)^(u+v) of the centre at pixel (N/2, N/2) (a
  library special case): pins the sign of the exponent, the axis each of u and
  v runs along and the phase centre.
- Shifting the image by one pixel multiplies every visibility by
  exp(-2 pi i u / N) (or v): pins the continuous (off-grid) coordinates.
- The adjoint with weights: Re <Phi x, W z> = <x, Re(Phi^H W z)>.
- k conjugate gradient iterations equal the textbook recurrence run with the
  dense Re(Phi^H W Phi) + rho I assembled from the pinned forward operator.
- Re(Phi^H W Phi) is Toeplitz: its entry (p, q) depends on p - q only (the
  structure the CUDA path's 2N convolution relies on).
- With every integer uv cell of the grid sampled once, Re(Phi^H Phi) = N^2 I and
  the problem is the circular one with PSF N delta and dirty image
  Re(Phi^H y) / N^2 * N: the visibility-mode ADMM equals the circular-mode ADMM,
  and the data-fit terms differ by the constant 1/2 ||y||^2 - 1/2 ||d||^2 / N^2.
- The history's objective is 1/2 sum w |y - Phi X|^2 plus the regularisers.
- With step I exact (CG run to convergence) He and Yuan's merit is monotone.
"""

import numpy as np
import pytest

import oracle
from oracle import daubechies
from paper_1504_06847_gb300 import synth
from tests import _dense

PRM = dict(mu_eps=0.003, mu_s=0.04, mu_nu=0.015, rho_P=0.7, rho_T=1.3, rho_V=1.9, rho_S=0.6)


def _random_problem(N=8, L=3, M=40, seed=1, integer=False, weights=True, cg_iters=4, J=2):
    rng = np.random.default_rng(seed)
    uv, vis, w = [], [], []
    for _ in range(L):
        if integer:
            q = rng.integers(-N // 2, N // 2, size=(M, 2)).astype(np.float64)
        else:
            q = rng.uniform(-0.49 * N, 0.49 * N, size=(M, 2))
        uv.append(q)
        vis.append(rng.normal(size=M) + 1j * rng.normal(size=M))
        w.append(rng.uniform(0.5, 1.5, size=M) if weights else np.ones(M))
    return oracle.Problem.visibilities(N, uv, vis, PRM, weights=w, J=J, cg_iters=cg_iters), uv, vis, w


def test_integer_coordinates_give_the_fft():
    N = 16
    pb, uv, _, _ = _random_problem(N=N, L=2, M=60, integer=True)
    x = np.random.default_rng(2).normal(size=(2, N, N))
    z = pb.apply_H(x)
    off = 0
    for l in range(2):
        F = np.fft.fft2(x[l])  # F[k_r, k_c] = sum x[r, c] e^{-2 pi i (k_r r + k_c c) / N}
        u, v = uv[l][:, 0].astype(int), uv[l][:, 1].astype(int)
        ref = F[v % N, u % N] * (-1.0) ** (u + v)
        assert np.max(np.abs(z[off:off + len(u)] - ref)) < 1e-11 * np.abs(F).max()
        off += len(u)


@pytest.mark.parametrize("axis", [0, 1])
def test_one_pixel_shift_is_a_phase(axis):
    N = 16
    pb, uv, _, _ = _random_problem(N=N, L=2, M=50)
    x = np.zeros((2, N, N))
    x[:, 2:N - 2, 2:N - 2] = np.random.default_rng(3).normal(size=(2, N - 4, N - 4))
    xs = np.roll(x, 1, axis=2 if axis == 0 else 1)  # column (u) or row (v) + 1, no wrap-around
    z, zs = pb.apply_H(x), pb.apply_H(xs)
    f = np.concatenate([q[:, axis] for q in uv])
    assert np.max(np.abs(zs - np.exp(-2j * np.pi * f / N) * z)) < 1e-11 * np.abs(z).max()


def test_adjoint_with_weights():
    pb, _, _, w = _random_problem(N=8, L=3, M=30)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 8, 8))
    z = rng.normal(size=90) + 1j * rng.normal(size=90)
    lhs = np.sum(np.concatenate(w) * np.real(np.conj(z) * pb.apply_H(x)))
    rhs = np.sum(x * pb.apply_H(z, adjoint=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # H^T y of the problem is the adjoint of its visibilities
    assert np.max(np.abs(pb.HtY - pb.apply_H(pb.y, adjoint=True))) < 1e-13 * np.abs(pb.HtY).max()


def _dense_normal(pb):
    """Re(Phi^H W Phi) of each band, column by column from the forward operator."""
    N, L = pb.N, pb.L
    A = np.zeros((L, N * N, N * N))
    for i in range(N * N):
        e = np.zeros((L, N, N))
        e[:, i // N, i % N] = 1.0
        A[:, :, i] = pb.apply_H(pb.apply_H(e), adjoint=True).reshape(L, -1)
    return A


def _dense_cg(Q, b, x, iters):
    r = b - Q @ x
    p = r.copy()
    g = r @ r
    for _ in range(iters):
        if g == 0.0:
            break
        q = Q @ p
        pq = p @ q
        if not pq > 0.0:
            break
        a = g / pq
        x = x + a * p
        r = r - a * q
        g2 = r @ r
        p = r + (g2 / g) * p
        g = g2
    return x


@pytest.mark.parametrize("iters", [1, 3, 10])
def test_cg_iterates_equal_the_textbook_recurrence(iters):
    pb, _, _, _ = _random_problem(N=8, L=2, M=45, seed=5)
    A = _dense_normal(pb)
    rng = np.random.default_rng(6)
    b = rng.normal(size=(2, 8, 8))
    x0 = rng.normal(size=(2, 8, 8))
    X = pb.solve(b, x0=x0, cg_iters=iters)
    for l in range(2):
        ref = _dense_cg(A[l] + pb.rho_bar * np.eye(64), b[l].ravel(), x0[l].ravel(), iters)
        assert np.max(np.abs(X[l].ravel() - ref)) < 1e-11 * max(1.0, np.abs(ref).max())


def test_normal_operator_is_toeplitz():
    pb, _, _, _ = _random_problem(N=8, L=1 + 1, M=35, seed=7)
    A = _dense_normal(pb)
    N = 8
    for l in range(2):
        seen = {}
        for p in range(N * N):
            for q in range(N * N):
                d = (p // N - q // N, p % N - q % N)
                if d in seen:
                    assert abs(A[l, p, q] - seen[d]) < 1e-11 * np.abs(A[l]).max()
                else:
                    seen[d] = A[l, p, q]
        assert np.allclose(A[l], A[l].T, atol=1e-12 * np.abs(A[l]).max())


def test_full_coverage_equals_the_circular_model():
    N, L = 8, 3
    rng = np.random.default_rng(8)
    ku, kv = np.meshgrid(np.arange(-N // 2, N // 2), np.arange(-N // 2, N // 2))
    cell = np.stack([ku.ravel(), kv.ravel()], axis=1).astype(np.float64)
    uv = [cell] * L
    vis = [rng.normal(size=N * N) + 1j * rng.normal(size=N * N) for _ in range(L)]
    vp = oracle.Problem.visibilities(N, uv, vis, PRM, J=2, cg_iters=2)
    d = vp.HtY
    psf = np.zeros((L, N, N))
    psf[:, N // 2, N // 2] = N
    cp = oracle.Problem(psf, d / N, PRM, J=2)
    a, Ha = vp.run(12, hist=True)
    b, Hb = cp.run(12, hist=True)
    for k in a:
        assert np.max(np.abs(a[k] - b[k])) < 1e-10 * max(1.0, np.abs(b[k]).max()), k
    const = 0.5 * sum(np.sum(np.abs(v) ** 2) for v in vis) - 0.5 * np.sum(d ** 2) / N ** 2
    assert np.max(np.abs((Ha[:, 3] - Hb[:, 3]) - const)) < 1e-9 * abs(const)
    for q in (0, 1, 2, 4, 5, 6):
        assert np.max(np.abs(Ha[:, q] - Hb[:, q])) <= 1e-9 * np.abs(Hb[:, q]).max() + 1e-300, q


def test_history_objective():
    pb, uv, vis, w = _random_problem(N=8, L=3, M=40, seed=9, J=2)
    st = pb.zero_state()
    for _ in range(3):
        h = pb.iterate(st, 1, hist=True)[0]
    X = st["X"]
    fit = 0.5 * np.sum(np.concatenate(w) * np.abs(pb.y - pb.apply_H(X)) ** 2)
    C = _dense.dct_matrix(pb.L)
    Ws = [_dense.dwt_matrix(hh, pb.N, 2) for _, hh in daubechies.dictionary(0x1FF)]
    l1s = sum(np.abs(Wk @ X[l].ravel()).sum() for Wk in Ws for l in range(pb.L))
    l1n = np.abs(np.einsum("kl,lij->kij", C, X)).sum()
    ref = fit + 0.5 * PRM["mu_eps"] * np.sum(X ** 2) + PRM["mu_s"] * l1s + PRM["mu_nu"] * l1n
    assert abs(h[3] - ref) < 1e-12 * ref


def test_merit_monotone_with_exact_step_I():
    c = synth.make_visibilities(16, 3, n_sources=2, n_antennas=10, seed=10, random_weights=True)
    pb = oracle.Problem.visibilities(16, c.uv, c.vis, synth.WORKLOAD_PARAMS, weights=c.weights, J=2, cg_iters=120)
    _, H = pb.run(20, hist=True)
    E = H[:, 2]
    assert np.all(E[2:] <= E[1:-1] * (1 + 1e-8) + 1e-20 * E[1]), E
    assert H[-1, 0] < 1e-2 * H[0, 0]


def test_synthetic_visibilities_follow_the_recipe():
    c = synth.make_visibilities(32, 4, n_sources=3, n_antennas=12, seed=11)
    assert len(c.uv) == 4 and all(len(q) == 66 for q in c.uv)  # 12 * 11 / 2 baselines
    for l, q in enumerate(c.uv):
        assert np.all(np.abs(q) < 0.4 * 32 + 1e-9)  # |p_i - p_j| <= 2, nu / nu0 <= 2, N / 10
        assert np.array_equal(q, q.astype(np.float32).astype(np.float64))
        assert abs(c.weights[l].sum() - 1.0) < 1e-12  # dirty beam peak 1
    # noise at 20 dB: the clean part is the oracle's forward operator
    pb = oracle.Problem.visibilities(32, c.uv, c.vis, PRM, J=2)
    clean = pb.apply_H(c.sky)
    noise = np.concatenate(c.vis) - clean
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(noise) ** 2))
    assert 17.0 < snr < 23.0
