"""FP64 CPU oracle of the spatio-spectral ADMM (arXiv:1504.06847, Algorithm 1).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library: its FFT, wavelet transform, DCT and filters are its own
(``mf_oracle.c`` and ``daubechies.py``).

Python-side helpers here only marshal numpy arrays into the C library, which
holds the arithmetic of every step.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import daubechies

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None
MAXF = 16
NHIST = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The oracle library; MF_ORACLE_LIB names another build of mf_oracle.c to
    load instead (the planted-mistake tests run the pins against mutants)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("MF_ORACLE_LIB")
            if not path:
                build()
                path = _LIB
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            c_int = ctypes.c_int
            L.orc_fft2.argtypes = [dp, dp, c_int, c_int, c_int]
            L.orc_dwt2.argtypes = [dp, dp, c_int, c_int, c_int, dp, c_int, c_int]
            L.orc_dct_matrix.argtypes = [c_int, dp]
            L.orc_setup.argtypes = [c_int, c_int, dp, dp, dp, dp, dp, dp, dp]
            L.orc_setup.restype = c_int
            L.orc_solve.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp, dp, dp, dp, dp]
            L.orc_solve.restype = c_int
            L.orc_make_b.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp] + [dp] * 8
            L.orc_make_b.restype = c_int
            L.orc_primal_dual.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp] + [dp] * 9
            L.orc_primal_dual.restype = c_int
            L.orc_iterate.argtypes = ([c_int, c_int, c_int, c_int, ip, dp, dp] + [dp] * 5 +
                                      [dp] * 9 + [c_int, dp])
            L.orc_iterate.restype = c_int
            L.orc_linear_setup.argtypes = [c_int, c_int, dp, dp, dp, dp, dp]
            L.orc_linear_setup.restype = c_int
            L.orc_linear_apply.argtypes = [c_int, c_int, dp, dp, dp, dp, c_int]
            L.orc_linear_apply.restype = None
            L.orc_solve_cg.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp, dp, dp, c_int, dp, dp]
            L.orc_solve_cg.restype = c_int
            L.orc_iterate_linear.argtypes = ([c_int, c_int, c_int, c_int, ip, dp, dp, dp, dp, dp, c_int, dp] +
                                             [dp] * 9 + [c_int, dp])
            L.orc_iterate_linear.restype = c_int
            L.orc_vis_setup.argtypes = [c_int, c_int, ip, dp, dp, dp, dp, dp, dp]
            L.orc_vis_setup.restype = c_int
            L.orc_vis_apply.argtypes = [c_int, c_int, ip, dp, dp, dp, dp, dp, dp, c_int]
            L.orc_vis_apply.restype = None
            L.orc_solve_cg_vis.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp, ip, dp, dp, dp, c_int, dp, dp]
            L.orc_solve_cg_vis.restype = c_int
            L.orc_iterate_vis.argtypes = ([c_int, c_int, c_int, c_int, ip, dp, dp, ip, dp, dp, dp, dp, dp, c_int,
                                           dp] + [dp] * 9 + [c_int, dp])
            L.orc_iterate_vis.restype = c_int
            _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------------------
# Transforms (exposed for the pins)
# ---------------------------------------------------------------------------

def fft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised 2-D DFT of each N x N image of x (complex128 [..., N, N])."""
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[-1]
    re = np.ascontiguousarray(x.real.reshape(-1, N, N))
    im = np.ascontiguousarray(x.imag.reshape(-1, N, N))
    lib().orc_fft2(_p(re), _p(im), N, re.shape[0], 1 if inverse else -1)
    return (re + 1j * im).reshape(x.shape)


def dwt2(x: np.ndarray, h: np.ndarray, J: int, inverse: bool = False) -> np.ndarray:
    """J-level periodic 2-D wavelet analysis (or synthesis) of each image."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    N = x.shape[-1]
    src = x.reshape(-1, N, N)
    out = np.empty_like(src)
    hh = np.zeros(MAXF)
    hh[: len(h)] = h
    lib().orc_dwt2(_p(src), _p(out), N, src.shape[0], J, _p(hh), len(h), -1 if inverse else 1)
    return out.reshape(x.shape)


def dct_matrix(L: int) -> np.ndarray:
    C = np.empty((L, L))
    lib().orc_dct_matrix(L, _p(C))
    return C


def chebyshev_matrix(L: int) -> np.ndarray:
    """The Chebyshev polynomial basis of Section 4 made orthonormal on the L
    equispaced bands: row k holds the degree-k polynomial of the family
    orthonormal on t_l = -1 + 2l/(L-1) (the discrete Chebyshev, or Gram,
    polynomials), with a positive leading coefficient.  Built by the
    Stieltjes procedure with full re-orthogonalisation: p_0 = 1/sqrt(L),
    p_k = t p_{k-1} minus its projections on p_0..p_{k-1}, normalised."""
    t = np.linspace(-1.0, 1.0, L)
    P = np.zeros((L, L))
    P[0] = 1.0 / np.sqrt(L)
    for k in range(1, L):
        q = t * P[k - 1]
        for _ in range(2):
            q = q - P[:k].T @ (P[:k] @ q)
        P[k] = q / np.linalg.norm(q)
    return P


SPECTRAL_BASES = {"dct": dct_matrix, "cheb": chebyshev_matrix}


# ---------------------------------------------------------------------------
# Problem and state
# ---------------------------------------------------------------------------

PARAM_ORDER = ("mu_eps", "mu_s", "mu_nu", "rho_P", "rho_T", "rho_V", "rho_S")


class Problem:
    """A cube (psf, y) with its regularisation, dictionary and level count.

    conv="circular" (the workloads): H is the circular convolution and step I
    the Fourier filter.  conv="linear": H is the linear ("same"-size)
    convolution by the PSF and step I runs cg_iters conjugate gradient
    iterations per band from the previous X."""

    def __init__(self, psf, y, params: dict, J: int = 3, mask: int = 0x1FF, bases=None, conv: str = "circular",
                 cg_iters: int = 0, spectral=("dct",)):
        self.psf = np.ascontiguousarray(psf, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.L, self.N = self.y.shape[0], self.y.shape[-1]
        assert self.psf.shape == self.y.shape == (self.L, self.N, self.N)
        self._common(params, J, mask, bases, spectral)
        shp = (self.L, self.N, self.N)
        if conv not in ("circular", "linear"):
            raise ValueError(conv)
        self.conv, self.cg_iters = conv, int(cg_iters)
        self.HtY = np.empty(shp)
        if conv == "linear":
            shp2 = (self.L, 2 * self.N, 2 * self.N)
            self.h2re, self.h2im = np.empty(shp2), np.empty(shp2)
            rc = lib().orc_linear_setup(self.N, self.L, _p(self.psf), _p(self.y), _p(self.h2re), _p(self.h2im),
                                        _p(self.HtY))
        else:
            self.hre, self.him = np.empty(shp), np.empty(shp)
            self.yre, self.yim = np.empty(shp), np.empty(shp)
            rc = lib().orc_setup(self.N, self.L, _p(self.psf), _p(self.y), _p(self.hre), _p(self.him),
                                 _p(self.yre), _p(self.yim), _p(self.HtY))
        assert rc == 0

    @classmethod
    def visibilities(cls, N: int, uv, vis, params: dict, weights=None, J: int = 3, mask: int = 0x1FF, bases=None,
                     cg_iters: int = 0, spectral=("dct",)):
        """The problem of Section 2's last paragraph: y_l are the visibilities
        vis[l] (complex [M_l]) sampled at uv[l] ([M_l, 2]: u, v in cells of the
        N x N image's Fourier grid) with weights[l] (default 1), and H_l maps
        the sky to them:
          (Phi_l x)_m = sum_{r,c} x[r][c] exp(-2 pi i (u_m (c - N/2) + v_m (r - N/2)) / N);
        the data fit is 1/2 sum_m w_m |y_m - (Phi_l x)_m|^2 and step I runs
        cg_iters conjugate gradient iterations on Re(Phi_l^H W Phi_l) + rho I."""
        self = cls.__new__(cls)
        self.L, self.N = len(uv), int(N)
        self._common(params, J, mask, bases, spectral)
        self.conv, self.cg_iters = "vis", int(cg_iters)
        counts = [len(np.asarray(a)) for a in uv]
        assert [len(np.asarray(a)) for a in vis] == counts
        self.voff = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        UV = np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1, 2) for a in uv])
        self.u, self.v = np.ascontiguousarray(UV[:, 0]), np.ascontiguousarray(UV[:, 1])
        if weights is None:
            self.w = np.ones(len(self.u))
        else:
            self.w = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64) for a in weights]))
        Y = np.concatenate([np.asarray(a, dtype=np.complex128) for a in vis])
        self.y = Y
        self.yre, self.yim = np.ascontiguousarray(Y.real), np.ascontiguousarray(Y.imag)
        self.psf = None
        self.HtY = np.empty((self.L, self.N, self.N))
        rc = lib().orc_vis_setup(self.N, self.L, _ip(self.voff), _p(self.u), _p(self.v), _p(self.w), _p(self.yre),
                                 _p(self.yim), _p(self.HtY))
        assert rc == 0
        return self

    def _vis_args(self):
        return (_ip(self.voff), _p(self.u), _p(self.v), _p(self.w))

    def _common(self, params, J, mask, bases, spectral):
        self.J = J
        self.bases = bases if bases is not None else daubechies.dictionary(mask)
        self.nb = len(self.bases)
        self.F = np.array([len(h) for _, h in self.bases], dtype=np.int32)
        self.h = np.zeros((self.nb, MAXF))
        for k, (_, h) in enumerate(self.bases):
            self.h[k, : len(h)] = h
        self.params = dict(params)
        # spectral dictionary W_nu: a union of m_nu orthonormal bases (step V divides by m_nu rho_V + rho_S)
        self.spectral = tuple(spectral)
        self.mnu = len(self.spectral)
        self.Cnu = [SPECTRAL_BASES[name](self.L) if isinstance(name, str) else np.asarray(name, dtype=np.float64)
                    for name in self.spectral]
        self.prm = np.concatenate([[float(self.params[k]) for k in PARAM_ORDER], [float(self.mnu)]] +
                                  [C.ravel() for C in self.Cnu])

    @property
    def rho_bar(self):
        p = self.params
        return p["mu_eps"] + p["rho_S"] + p["rho_P"] + self.nb * p["rho_T"]

    def _hdr(self):
        return (self.N, self.L, self.J, self.nb, _ip(self.F), _p(self.h), _p(self.prm))

    def zero_state(self) -> dict:
        shp = (self.L, self.N, self.N)
        st = {k: np.zeros(shp) for k in ("X", "P", "S", "GP", "GS")}
        vshp = shp if self.mnu == 1 else (self.mnu,) + shp
        st["V"] = np.zeros(vshp)
        st["GV"] = np.zeros(vshp)
        st["T"] = np.zeros((self.nb,) + shp)
        st["GT"] = np.zeros((self.nb,) + shp)
        return st

    def iterate(self, state: dict, n_iter: int, hist: bool = False):
        """Run Algorithm 1 for n_iter iterations, updating `state` in place.
        Returns the per-iteration history array [n_iter, NHIST] (or None)."""
        H = np.zeros((n_iter, NHIST)) if hist else None
        s = state
        arrays = [_p(s[k]) for k in ("X", "P", "T", "V", "S", "GP", "GT", "GV", "GS")]
        hp = _p(H) if hist else ctypes.POINTER(ctypes.c_double)()
        if self.conv == "linear":
            rc = lib().orc_iterate_linear(*self._hdr(), _p(self.h2re), _p(self.h2im), _p(self.y), self.cg_iters,
                                          _p(self.HtY), *arrays, int(n_iter), hp)
        elif self.conv == "vis":
            rc = lib().orc_iterate_vis(*self._hdr(), *self._vis_args(), _p(self.yre), _p(self.yim), self.cg_iters,
                                       _p(self.HtY), *arrays, int(n_iter), hp)
        else:
            rc = lib().orc_iterate(*self._hdr(), _p(self.hre), _p(self.him), _p(self.yre),
                                   _p(self.yim), _p(self.HtY), *arrays, int(n_iter), hp)
        assert rc == 0
        return H

    def run(self, n_iter: int, hist: bool = False):
        st = self.zero_state()
        H = self.iterate(st, n_iter, hist)
        return st, H

    def solve(self, b: np.ndarray, x0: np.ndarray | None = None, cg_iters: int | None = None) -> np.ndarray:
        """Step I alone, b the full right-hand side of Eq. matB: X = Q^-1 b by the
        Fourier filter (circular H), or cg_iters conjugate gradient iterations
        from x0 (default 0) for the linear H."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if self.conv in ("linear", "vis"):
            X = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, order="C")
            it = self.cg_iters if cg_iters is None else int(cg_iters)
            if self.conv == "vis":
                rc = lib().orc_solve_cg_vis(*self._hdr(), *self._vis_args(), it, _p(b), _p(X))
            else:
                rc = lib().orc_solve_cg(*self._hdr(), _p(self.h2re), _p(self.h2im), it, _p(b), _p(X))
        else:
            X = np.empty_like(b)
            rc = lib().orc_solve(*self._hdr(), _p(self.hre), _p(self.him), _p(b), _p(X))
        assert rc == 0
        return X

    def apply_H(self, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """H x (or H^T x) of the linear convolution, for every band.  For the
        visibility operator: Phi x (x a real cube; returns the concatenated
        complex visibilities) or, adjoint, Re(Phi^H W x) (x complex visibilities)."""
        if self.conv == "vis":
            n = int(self.voff[-1])
            if adjoint:
                z = np.asarray(x, dtype=np.complex128)
                zre, zim = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
                out = np.empty((self.L, self.N, self.N))
                lib().orc_vis_apply(self.N, self.L, *self._vis_args(), _p(out), _p(zre), _p(zim), 1)
                return out
            xc = np.ascontiguousarray(x, dtype=np.float64)
            zre, zim = np.empty(n), np.empty(n)
            lib().orc_vis_apply(self.N, self.L, *self._vis_args(), _p(xc), _p(zre), _p(zim), 0)
            return zre + 1j * zim
        assert self.conv == "linear"
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(x)
        lib().orc_linear_apply(self.N, self.L, _p(self.h2re), _p(self.h2im), _p(x), _p(out), int(adjoint))
        return out

    def make_b(self, st: dict) -> np.ndarray:
        """Eq. matB from a state."""
        b = np.empty((self.L, self.N, self.N))
        rc = lib().orc_make_b(*self._hdr(), _p(self.HtY), _p(st["P"]), _p(st["T"]), _p(st["S"]),
                              _p(st["GP"]), _p(st["GT"]), _p(st["GS"]), _p(b))
        assert rc == 0
        return b

    def primal_dual(self, X: np.ndarray, st: dict) -> None:
        """Steps II-VI in place on `st` for a given new X (st['X'] is set to X)."""
        st["X"][...] = X
        rc = lib().orc_primal_dual(*self._hdr(), _p(st["X"]), _p(st["P"]), _p(st["T"]),
                                   _p(st["V"]), _p(st["S"]), _p(st["GP"]), _p(st["GT"]),
                                   _p(st["GV"]), _p(st["GS"]))
        assert rc == 0


# ---------------------------------------------------------------------------
# Spectral-index fit (post-processing of the paper's first simulation, Section 4)
# ---------------------------------------------------------------------------

def spectral_index(cube: np.ndarray, nu, nu0: float | None = None, floor: float = 0.0):
    """Per-pixel least-squares fit of log S(nu) = c + alpha u + beta u^2,
    u = log(nu / nu0), over the bands of cube [L, N, N] (FP64, numpy lstsq).
    Pixels with any S <= floor get NaN.  Returns (c, alpha, beta), each [N, N]."""
    cube = np.asarray(cube, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    L, N = cube.shape[0], cube.shape[-1]
    u = np.log(nu / (nu[0] if nu0 is None else nu0))
    A = np.stack([np.ones(L), u, u * u], axis=1)
    ok = np.all(cube > floor, axis=0)
    logs = np.log(np.where(cube > 0, cube, 1.0)).reshape(L, N * N)
    coef = np.linalg.lstsq(A, logs, rcond=None)[0].reshape(3, N, N)
    coef[:, ~ok] = np.nan
    return coef[0], coef[1], coef[2]
