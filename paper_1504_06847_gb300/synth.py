"""Seeded synthetic wide-band radio-interferometric cubes.

Stand-ins for the MeerKAT/MeqTrees PSFs and sky images of the paper's
Section 4 (which are not available): a sky of elliptical Gaussian sources
with curved power-law spectra, a per-band PSF built from a random disk array
whose baselines scale with frequency, and a dirty cube ``y_l = H_l x_l + n``
(the narrow-band model ``nbmodel`` of Section 2) with white Gaussian noise of
one variance for the whole cube at a given SNR (Section 4, M31 test: 20 dB).

This module only simulates observations.  It holds none of the
reconstruction method's arithmetic and imports neither the CUDA binding nor
the oracle, so both sides can draw the same inputs from it.

Recipe (all draws from ``numpy.random.default_rng(seed)`` in this order):

1. frequencies ``nu_l = 1.0 + l/(L-1)`` GHz, ``nu_0 = 1.0`` GHz;
2. per source: centre ~ U[0.1N, 0.9N]^2, sigma_major, sigma_minor ~ U(1, 6) px,
   angle ~ U(0, pi), peak S0 ~ U(0.1, 1.0), alpha ~ U(-1, 0.5),
   beta ~ U(-0.2, 0.2); spectrum ``S0 (nu/nu0)^(alpha + beta ln(nu/nu0))``;
   the last ``round(point_frac * n_sources)`` sources are single pixels;
3. antennas uniform in the unit disk (r = sqrt(U), theta ~ U(0, 2 pi));
   for every ordered pair i != j the uv cell
   ``round((p_i - p_j) * (nu_l/nu_0) * N/10) mod N`` and the cell (0, 0) are
   set in a binary mask; ``psf = Re(ifft2(mask))`` normalised to peak 1 and
   shifted so that the peak sits at pixel (N/2, N/2);
4. ``y_l = psf_l (circularly convolved) x_l + n``, ``n ~ N(0, sigma^2)`` with
   ``sigma = rms(Hx) * 10^(-snr_db/20)``.

Visibility-domain observations (``make_visibilities``, the measurement model of
Section 2's last paragraph): the same sky and array draws, then per band one
visibility per unordered baseline i < j at the continuous uv point
``(p_i - p_j) * (nu_l/nu_0) * N/10`` (cells; rounded to float32 so that every
consumer sees the same coordinates), the exact sum
``sum_{r,c} x[r][c] exp(-2 pi i (u (c - N/2) + v (r - N/2)) / N)`` plus complex
white noise (each part of standard deviation ``sigma/sqrt(2)``,
``sigma = rms|Phi x| * 10^(-snr_db/20)``), and weights 1 or, with
``random_weights``, ``U(0.5, 1.5)``, divided by their sum in each band, so that
the dirty beam ``sum_m w_m exp(2 pi i u_m . d / N)`` peaks at 1 like the PSF of
step 3 (and ``Re(Phi^H W Phi) + rho I`` stays as well conditioned as in the
image-domain workloads).
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Cube:
    sky: np.ndarray  # [L][N][N] float64, the synthetic truth (>= 0)
    psf: np.ndarray  # [L][N][N] float64, peak 1 at (N/2, N/2)
    y: np.ndarray  # [L][N][N] float64, dirty cube
    nu: np.ndarray  # [L] GHz
    sigma: float  # noise standard deviation


def _gaussian_patch(N, cx, cy, smaj, smin, ang):
    half = int(np.ceil(6.0 * smaj)) + 1
    ix = np.arange(int(np.floor(cx)) - half, int(np.floor(cx)) + half + 2)
    iy = np.arange(int(np.floor(cy)) - half, int(np.floor(cy)) + half + 2)
    dx = ix[None, :] - cx
    dy = iy[:, None] - cy
    c, s = np.cos(ang), np.sin(ang)
    u = c * dx + s * dy
    v = -s * dx + c * dy
    g = np.exp(-0.5 * ((u / smaj) ** 2 + (v / smin) ** 2))
    return np.mod(iy, N), np.mod(ix, N), g


def make_cube(N: int, L: int, n_sources: int, n_antennas: int, seed: int,
              point_frac: float = 0.0, snr_db: float = 20.0) -> Cube:
    if L < 2:
        raise ValueError("L must be >= 2")
    rng = np.random.default_rng(seed)
    nu = 1.0 + np.arange(L) / (L - 1)
    nu0 = 1.0
    sky = _sky(N, L, n_sources, rng, nu, nu0, point_frac)
    return observe(sky, nu, nu0, n_antennas, rng, snr_db)


@dataclasses.dataclass
class Visibilities:
    sky: np.ndarray  # [L][N][N] float64, the synthetic truth (>= 0)
    uv: list  # L arrays [M_l, 2] float64 (float32-representable), (u, v) in cells
    vis: list  # L arrays [M_l] complex128
    weights: list  # L arrays [M_l] float64
    nu: np.ndarray  # [L] GHz
    sigma: float  # noise standard deviation (complex)


def make_visibilities(N: int, L: int, n_sources: int, n_antennas: int, seed: int, snr_db: float = 20.0,
                      random_weights: bool = False, point_frac: float = 0.0) -> Visibilities:
    """The recipe's sky and array, observed as visibilities (see the module docstring)."""
    if L < 2:
        raise ValueError("L must be >= 2")
    rng = np.random.default_rng(seed)
    nu = 1.0 + np.arange(L) / (L - 1)
    nu0 = 1.0
    sky = _sky(N, L, n_sources, rng, nu, nu0, point_frac)
    r = np.sqrt(rng.uniform(0.0, 1.0, size=n_antennas))
    th = rng.uniform(0.0, 2.0 * np.pi, size=n_antennas)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    i, j = np.triu_indices(n_antennas, k=1)
    base = pos[i] - pos[j]
    uvs, clean = [], []
    n = np.arange(N) - N // 2
    for l in range(L):
        uv = (base * (nu[l] / nu0) * N / 10.0).astype(np.float32).astype(np.float64)
        eu = np.exp(-2j * np.pi * np.outer(uv[:, 0], n) / N)  # [M, N] along columns
        ev = np.exp(-2j * np.pi * np.outer(uv[:, 1], n) / N)  # [M, N] along rows
        clean.append(np.einsum("mr,mr->m", ev, eu @ sky[l].T))
        uvs.append(uv)
    allv = np.concatenate(clean)
    sigma = float(np.sqrt(np.mean(np.abs(allv) ** 2)) * 10.0 ** (-snr_db / 20.0))
    vis = [v + rng.normal(0.0, sigma / np.sqrt(2), size=v.shape) + 1j * rng.normal(0.0, sigma / np.sqrt(2),
                                                                                     size=v.shape)
           for v in clean]
    if random_weights:
        weights = [rng.uniform(0.5, 1.5, size=len(v)) for v in vis]
    else:
        weights = [np.ones(len(v)) for v in vis]
    weights = [a / a.sum() if len(a) else a for a in weights]
    return Visibilities(sky=sky, uv=uvs, vis=vis, weights=weights, nu=nu, sigma=sigma)


def _sky(N, L, n_sources, rng, nu, nu0, point_frac):
    """Step 2 of the recipe: the sky cube [L][N][N]."""
    lognu = np.log(nu / nu0)

    sky = np.zeros((L, N, N))
    n_point = int(round(point_frac * n_sources))
    for s in range(n_sources):
        cx, cy = rng.uniform(0.1 * N, 0.9 * N, size=2)
        smaj, smin = np.sort(rng.uniform(1.0, 6.0, size=2))[::-1]
        ang = rng.uniform(0.0, np.pi)
        s0 = rng.uniform(0.1, 1.0)
        alpha = rng.uniform(-1.0, 0.5)
        beta = rng.uniform(-0.2, 0.2)
        spec = s0 * np.exp((alpha + beta * lognu) * lognu)
        if s >= n_sources - n_point:
            sky[:, int(cy) % N, int(cx) % N] += spec
        else:
            ry, rx, g = _gaussian_patch(N, cx, cy, smaj, smin, ang)
            if len(ry) <= N and len(rx) <= N:
                sky[:, ry[:, None], rx[None, :]] += spec[:, None, None] * g[None]
            else:  # the patch is wider than the image and wraps onto itself
                img = np.zeros((N, N))
                np.add.at(img, (ry[:, None], rx[None, :]), g)
                sky += spec[:, None, None] * img[None]
    return sky


def observe(sky: np.ndarray, nu: np.ndarray, nu0: float, n_antennas: int, rng, snr_db: float = 20.0) -> Cube:
    """Steps 3-4 of the recipe for a given sky [L][N][N] at frequencies nu (GHz):
    the disk array drawn from rng, the per-band PSFs (baselines scaled by
    nu/nu0) and the dirty cube with white noise at snr_db."""
    L, N = sky.shape[0], sky.shape[-1]
    r = np.sqrt(rng.uniform(0.0, 1.0, size=n_antennas))
    th = rng.uniform(0.0, 2.0 * np.pi, size=n_antennas)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    diff = pos[:, None, :] - pos[None, :, :]
    off = ~np.eye(n_antennas, dtype=bool)
    diff = diff[off]  # ordered pairs i != j

    psf = np.empty((L, N, N))
    for l in range(L):
        uv = np.mod(np.rint(diff * (nu[l] / nu0) * N / 10.0).astype(np.int64), N)
        mask = np.zeros((N, N))
        mask[uv[:, 1], uv[:, 0]] = 1.0
        mask[0, 0] = 1.0
        p = np.real(np.fft.ifft2(mask))
        p /= p[0, 0]
        psf[l] = np.fft.fftshift(p)

    # circular convolution with the PSF centred at (N/2, N/2)
    hx = np.real(np.fft.ifft2(np.fft.fft2(sky) * np.fft.fft2(np.fft.ifftshift(psf, axes=(1, 2)))))
    sigma = float(np.sqrt(np.mean(hx ** 2)) * 10.0 ** (-snr_db / 20.0))
    y = hx + rng.normal(0.0, sigma, size=hx.shape)
    return Cube(sky=sky, psf=psf, y=y, nu=nu, sigma=sigma)


# Workloads used by the tests and the benchmark (name -> generator arguments).
WORKLOADS = {
    "64x64x8": dict(N=64, L=8, n_sources=6, n_antennas=64, seed=1),
    "256x256x32": dict(N=256, L=32, n_sources=40, n_antennas=256, seed=2),
    "1024x1024x64": dict(N=1024, L=64, n_sources=300, n_antennas=512, seed=3, point_frac=0.2),
}

# Regularisation and penalty values of the workloads above: mu_eps from the
# paper's Section 4 settings, mu_s, mu_nu and one rho for all four penalties.
WORKLOAD_PARAMS = dict(mu_eps=0.001, mu_s=0.05, mu_nu=0.01,
                       rho_P=1.0, rho_T=1.0, rho_V=1.0, rho_S=1.0)

# The paper's own settings (Section 4), and its fixed iteration count (it
# stops after 350 iterations instead of testing the residuals).
PAPER_PARAMS = dict(mu_eps=0.001, mu_s=0.5, mu_nu=1.0,
                    rho_P=1.0, rho_T=5.0, rho_V=2.0, rho_S=1.0)
PAPER_ITERS = 350


def asymmetric_psf(psf: np.ndarray, seed: int, depth: float = 0.3) -> np.ndarray:
    """The PSF cube multiplied pixel by pixel by 1 + depth U(-1, 1): the same
    scale, no point symmetry about (N/2, N/2).  The recipe's PSFs are
    point-symmetric (every uv cell comes with its mirror), for which H^T = H;
    this variant makes the transposed operator differ from H."""
    rng = np.random.default_rng(seed)
    return psf * (1.0 + depth * rng.uniform(-1.0, 1.0, size=psf.shape))


def workload(name: str) -> Cube:
    return make_cube(**WORKLOADS[name])


def batch_shapes(count: int = 16, seed: int = 400):
    """Uneven (N, L) shapes of the batched form: N in {128, 256, 512}, L in {16, 32, 64}."""
    rng = np.random.default_rng(seed)
    return [(int(rng.choice([128, 256, 512])), int(rng.choice([16, 32, 64]))) for _ in range(count)]


def batch_workload(count: int = 16, seed: int = 400, n_antennas: int = 256):
    """The cubes of the batched form: cube i has shape batch_shapes()[i], seed seed + i
    and 40 (N/256)^2 sources."""
    return [make_cube(N, L, n_sources=max(2, int(40 * (N / 256) ** 2)), n_antennas=n_antennas, seed=seed + i)
            for i, (N, L) in enumerate(batch_shapes(count, seed))]



def two_gaussians(N: int = 256, L: int = 15, sigma_px: float = 12.0, n_antennas: int = 64, seed: int = 108,
                  snr_db: float = 20.0) -> Cube:
    """The two-Gaussian sky of the paper's first simulation (Section 4): two
    overlapping Gaussian profiles centred at pixels 108 and 148 of the middle
    row (of a 256-pixel image; scaled with N), peak 1 at the first band, with
    constant spectral indices -1 and +1, over L bands from 1.025 GHz in 50 MHz
    steps (nu0 = 1.025 GHz), observed with the disk-array PSFs of the recipe.
    The paper gives no width: sigma_px (12 px) makes the profiles overlap
    (each is at a quarter of its peak at the midpoint)."""
    rng = np.random.default_rng(seed)
    nu = 1.025 + 0.05 * np.arange(L)
    nu0 = float(nu[0])
    centres = [(N // 2, 108.0 * N / 256.0, -1.0), (N // 2, 148.0 * N / 256.0, 1.0)]
    yy, xx = np.mgrid[0:N, 0:N]
    sky = np.zeros((L, N, N))
    for cy, cx, alpha in centres:
        g = np.exp(-0.5 * (((yy - cy) ** 2 + (xx - cx) ** 2) / sigma_px ** 2))
        sky += (nu / nu0)[:, None, None] ** alpha * g[None]
    return observe(sky, nu, nu0, n_antennas, rng, snr_db)
