"""GB300 (sm_103a) spatio-spectral ADMM deconvolution (arXiv:1504.06847).

Thin ctypes binding of the C ABI in ``include/mf.h``.  Every step of the
iteration runs in the library's CUDA kernels; PyTorch only provides device
memory (tensors whose pointers are passed through) and streams.  There is no
CPU fallback: importing the binding without the built library raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmf.so")

MF_OK, MF_ERR_INVALID, MF_ERR_OOM, MF_ERR_CUDA, MF_ERR_TIMEOUT, MF_ERR_NONFINITE, MF_ERR_TOO_LARGE = range(7)
XSTEP_NOALLOC_MAX_VOXELS = 1 << 19
MF_FP32, MF_FP64, MF_FP32_DCT_SPLITBF16 = range(3)
ARR_X, ARR_GAMMA_P, ARR_S_DCT, ARR_GAMMA_V, ARR_GAMMA_S_DCT, ARR_B, ARR_GAMMA_T, ARR_GAMMA_V2, ARR_HTY = range(9)
SPECTRAL_DCT, SPECTRAL_CHEBYSHEV = 0, 1

EXPORTS = ["mf_params_default", "mf_plan_create", "mf_plan_create_f64", "mf_plan_destroy",
           "mf_plan_device_bytes", "mf_admm_iterate", "mf_admm_iterate_f64", "mf_plan_get_array",
           "mf_plan_set_array", "mf_plan_get_state", "mf_plan_set_state", "mf_plan_get_report",
           "mf_wavelet_filter", "mf_status_string", "mf_plan_set_timing", "mf_plan_get_timing",
           "mf_kernel_name", "mf_xstep_noalloc", "mf_plan_set_option", "mf_batch_iterate",
           "mf_admm_backward", "mf_plan_clear_status", "mf_spectral_index", "mf_plan_create_linear",
           "mf_spectral_basis", "mf_plan_create_vis", "mf_vis_predict"]
MF_OPT_WAV_TILE, MF_OPT_TEST_TC_STALL = 0, 1

KERNELS = ["rows_fwd", "cols_solve", "rows_inv", "spectral", "wav_ll", "wav_level1", "wav_levelj", "setup",
           "reduce", "dual", "cg"]


class MFError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class Params(ctypes.Structure):
    _fields_ = [("mu_eps", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_nu", ctypes.c_double),
                ("rho_P", ctypes.c_double), ("rho_T", ctypes.c_double), ("rho_V", ctypes.c_double),
                ("rho_S", ctypes.c_double), ("wavelet_levels", ctypes.c_int),
                ("wavelet_mask", ctypes.c_uint), ("precision", ctypes.c_int),
                ("resid_every", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("cg_iters", ctypes.c_int),
                ("spectral_mask", ctypes.c_uint)]


class Report(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int), ("resid_iter", ctypes.c_int),
                ("primal_res", ctypes.c_double), ("dual_gamma", ctypes.c_double),
                ("objective", ctypes.c_double), ("x_min", ctypes.c_double),
                ("x_norm2", ctypes.c_double), ("dual_res", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmf.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        L.mf_params_default.argtypes = [ctypes.POINTER(Params)]
        L.mf_params_default.restype = None
        for name in ("mf_plan_create", "mf_plan_create_f64", "mf_plan_create_linear"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
            f.restype = ctypes.c_int
        L.mf_plan_create_vis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp, vp,
                                         ctypes.POINTER(vp)]
        L.mf_plan_create_vis.restype = ctypes.c_int
        L.mf_vis_predict.argtypes = [vp, vp, vp, vp]
        L.mf_vis_predict.restype = ctypes.c_int
        L.mf_plan_destroy.argtypes = [vp]
        L.mf_plan_destroy.restype = None
        L.mf_plan_device_bytes.argtypes = [vp]
        L.mf_plan_device_bytes.restype = sz
        for name in ("mf_admm_iterate", "mf_admm_iterate_f64"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, ctypes.POINTER(Params), ctypes.c_int]
            f.restype = ctypes.c_int
        L.mf_plan_get_array.argtypes = [vp, ctypes.c_int, vp, ctypes.POINTER(sz)]
        L.mf_plan_get_array.restype = ctypes.c_int
        L.mf_plan_set_array.argtypes = [vp, ctypes.c_int, vp, sz]
        L.mf_plan_set_array.restype = ctypes.c_int
        L.mf_plan_get_state.argtypes = [vp, vp, ctypes.POINTER(sz)]
        L.mf_plan_get_state.restype = ctypes.c_int
        L.mf_plan_set_state.argtypes = [vp, vp, sz]
        L.mf_plan_set_state.restype = ctypes.c_int
        L.mf_plan_get_report.argtypes = [vp, ctypes.POINTER(Report)]
        L.mf_plan_get_report.restype = ctypes.c_int
        L.mf_spectral_basis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.mf_spectral_basis.restype = ctypes.c_int
        L.mf_wavelet_filter.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        L.mf_wavelet_filter.restype = ctypes.c_int
        L.mf_status_string.argtypes = [ctypes.c_int]
        L.mf_status_string.restype = ctypes.c_char_p
        L.mf_plan_set_timing.argtypes = [vp, ctypes.c_int]
        L.mf_plan_set_timing.restype = ctypes.c_int
        L.mf_plan_get_timing.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong)]
        L.mf_plan_get_timing.restype = ctypes.c_int
        L.mf_kernel_name.argtypes = [ctypes.c_int]
        L.mf_kernel_name.restype = ctypes.c_char_p
        L.mf_batch_iterate.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(Params),
                                       ctypes.c_int]
        L.mf_batch_iterate.restype = ctypes.c_int
        L.mf_admm_backward.argtypes = [vp, vp, ctypes.POINTER(Params), ctypes.c_int, vp, vp,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        L.mf_admm_backward.restype = ctypes.c_int
        L.mf_plan_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.mf_plan_set_option.restype = ctypes.c_int
        L.mf_spectral_index.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_double, ctypes.c_float, vp, vp, vp, vp]
        L.mf_spectral_index.restype = ctypes.c_int
        L.mf_plan_clear_status.argtypes = [vp]
        L.mf_plan_clear_status.restype = ctypes.c_int
        L.mf_xstep_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(Params), vp]
        L.mf_xstep_noalloc.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().mf_status_string(int(s)).decode()


def _check(rc, what):
    if rc != MF_OK:
        raise MFError(rc, what)


def default_params(**kw) -> Params:
    p = Params()
    lib().mf_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def wavelet_filter(K: int):
    """The library's DbK low-pass taps (host doubles)."""
    taps = (ctypes.c_double * 16)()
    n = ctypes.c_int()
    _check(lib().mf_wavelet_filter(K, taps, ctypes.byref(n)), "mf_wavelet_filter")
    return [taps[i] for i in range(n.value)]


def spectral_basis(kind: int, L: int):
    """The library's L x L spectral basis (SPECTRAL_DCT or SPECTRAL_CHEBYSHEV), host doubles,
    as a list of rows."""
    out = (ctypes.c_double * (L * L))()
    _check(lib().mf_spectral_basis(int(kind), int(L), out), "mf_spectral_basis")
    return [[out[k * L + l] for l in range(L)] for k in range(L)]


def batch_iterate(plans, ys, n_iter: int, **kw):
    """Batched form: n_iter iterations of every (plan, y) pair in one CUDA graph
    launch (see mf_batch_iterate).  FP32 plans; ys are CUDA tensors [L, N, N]."""
    import torch

    if len(plans) != len(ys) or not plans:
        raise ValueError("one dirty cube per plan")
    for p_, y in zip(plans, ys):
        if p_.dtype != torch.float32:
            raise ValueError("the batched form takes FP32 plans")
        if y.dtype != torch.float32 or not y.is_cuda or tuple(y.shape) != (p_.L, p_.N, p_.N):
            raise ValueError("each y must be a float32 CUDA tensor matching its plan")
    ys = [y.contiguous() for y in ys]
    if "stream" not in kw:
        kw["stream"] = torch.cuda.current_stream(ys[0].device).cuda_stream
    prm = default_params(**kw)
    hp = (ctypes.c_void_p * len(plans))(*[p_._h.value for p_ in plans])
    yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    _check(lib().mf_batch_iterate(hp, yp, len(plans), ctypes.byref(prm), int(n_iter)), "mf_batch_iterate")
    for p_, y in zip(plans, ys):
        p_._y_keepalive = y


def spectral_index(cube, nu, nu0=None, floor=0.0, stream=None):
    """Per-pixel fit log S = c + alpha u + beta u^2, u = log(nu/nu0), of a float32
    CUDA cube [L, N, N] (see mf_spectral_index).  nu: L frequencies; nu0
    defaults to nu[0].  Returns (c, alpha, beta) as float32 CUDA tensors [N, N]
    (NaN where some S(nu_l) <= floor)."""
    import torch

    if cube.dtype != torch.float32 or not cube.is_cuda or cube.dim() != 3 or cube.shape[1] != cube.shape[2]:
        raise ValueError("cube must be a float32 CUDA tensor [L, N, N]")
    cube = cube.contiguous()
    L_, N_ = int(cube.shape[0]), int(cube.shape[1])
    if len(nu) != L_:
        raise ValueError("one frequency per band")
    nu_c = (ctypes.c_double * L_)(*[float(v) for v in nu])
    nu0 = float(nu[0] if nu0 is None else nu0)
    outs = [torch.empty((N_, N_), dtype=torch.float32, device=cube.device) for _ in range(3)]
    with torch.cuda.device(cube.device):
        s = torch.cuda.current_stream(cube.device).cuda_stream if stream is None else stream
        _check(lib().mf_spectral_index(N_, L_, ctypes.c_void_p(cube.data_ptr()), nu_c, nu0, float(floor),
                                       *[ctypes.c_void_p(o.data_ptr()) for o in outs], ctypes.c_void_p(s)),
               "mf_spectral_index")
    return tuple(outs)


def xstep_noalloc(psf, y, b, x_out, **kw):
    """Step I, x = (H^T H + rho I)^-1 (H^T y + b), without any device allocation
    (the library's static scratch; see mf_xstep_noalloc in include/mf.h).  For
    callers that cannot allocate device memory: all arguments are existing
    float32 CUDA tensors [L, N, N]; x_out receives the result.  Enqueued on the
    current stream unless ``stream`` is given."""
    import torch

    L_, N_ = int(y.shape[0]), int(y.shape[-1])
    for t in (psf, y, b, x_out):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (L_, N_, N_):
            raise ValueError("psf, y, b, x_out must be contiguous float32 CUDA tensors [L, N, N]")
        if t.device != y.device:
            raise ValueError("psf, y, b, x_out must be on one device")
    # the library uses the static array and launches on the current device
    with torch.cuda.device(y.device):
        if "stream" not in kw:
            kw["stream"] = torch.cuda.current_stream(y.device).cuda_stream
        p = default_params(**kw)
        _check(lib().mf_xstep_noalloc(N_, L_, ctypes.c_void_p(psf.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(b.data_ptr()), ctypes.byref(p),
                                      ctypes.c_void_p(x_out.data_ptr())), "mf_xstep_noalloc")


class Plan:
    """A plan for N x N x L cubes on the current CUDA device.

    psf: CUDA tensor [L, N, N] (float32, or float64 for an FP64 plan).
    linear=True: H is the linear (zero-padded, non-circulant) convolution and
    step I runs conjugate gradients (float32; see mf_plan_create_linear).
    Plan.from_visibilities: H maps the sky to sampled visibilities (see
    mf_plan_create_vis); iterate() then takes the visibilities.
    """

    n_vis = None

    @classmethod
    def from_visibilities(cls, N: int, uv, weights=None):
        """uv: list of L CUDA float32 tensors [M_l, 2] ((u, v) in cells of the
        N x N image's Fourier grid); weights: list of L CUDA float32 tensors
        [M_l] or None (all 1).  The plan copies both."""
        import torch

        self = cls.__new__(cls)
        self.L, self.N = len(uv), int(N)
        self.dtype = torch.float32
        self.device = uv[0].device
        counts = [int(a.shape[0]) for a in uv]
        self.n_vis = sum(counts)
        cat = torch.cat([a.reshape(-1, 2) for a in uv]).to(torch.float32).contiguous()
        if not cat.is_cuda:
            raise ValueError("uv must be CUDA tensors")
        wc = None
        if weights is not None:
            wc = torch.cat([a.reshape(-1) for a in weights]).to(torch.float32).contiguous()
            if wc.shape[0] != self.n_vis or not wc.is_cuda:
                raise ValueError("weights must match uv")
        c_counts = (ctypes.c_int * self.L)(*counts)
        h = ctypes.c_void_p()
        _check(lib().mf_plan_create_vis(self.N, self.L, c_counts, ctypes.c_void_p(cat.data_ptr()),
                                        ctypes.c_void_p(wc.data_ptr()) if wc is not None else None,
                                        ctypes.byref(h)), "mf_plan_create_vis")
        self._h = h
        return self

    def predict(self, x=None):
        """Model visibilities Phi x of a visibility plan (see mf_vis_predict): x a
        float32 CUDA tensor [L, N, N] or None for the plan's X; returns complex64
        [sum M_l] in the plan's visibility order."""
        import torch

        if self.n_vis is None:
            raise ValueError("predict needs a plan from Plan.from_visibilities")
        if x is not None:
            if x.dtype != torch.float32 or not x.is_cuda or tuple(x.shape) != (self.L, self.N, self.N):
                raise ValueError("x must be a float32 CUDA tensor [L, N, N]")
            x = x.contiguous()
        out = torch.empty((self.n_vis, 2), dtype=torch.float32, device=self.device)
        s = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib().mf_vis_predict(self._h, ctypes.c_void_p(x.data_ptr()) if x is not None else None,
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s)), "mf_vis_predict")
        self._x_keepalive = x
        return torch.view_as_complex(out)

    def __init__(self, psf, linear: bool = False):
        import torch

        if not psf.is_cuda or psf.dim() != 3 or psf.shape[1] != psf.shape[2]:
            raise ValueError("psf must be a CUDA tensor [L, N, N]")
        self.dtype = psf.dtype
        if self.dtype not in (torch.float32, torch.float64):
            raise ValueError("psf must be float32 or float64")
        self.L, self.N = int(psf.shape[0]), int(psf.shape[1])
        psf = psf.contiguous()
        h = ctypes.c_void_p()
        if linear and self.dtype != torch.float32:
            raise ValueError("linear-convolution plans are float32")
        create = (lib().mf_plan_create_linear if linear else
                  lib().mf_plan_create if self.dtype == torch.float32 else lib().mf_plan_create_f64)
        _check(create(self.N, self.L, ctypes.c_void_p(psf.data_ptr()), ctypes.byref(h)), "mf_plan_create")
        self._h = h
        self.device = psf.device

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return int(lib().mf_plan_device_bytes(self._h))

    def params(self, **kw) -> Params:
        import torch

        kw.setdefault("precision", MF_FP32 if self.dtype == torch.float32 else MF_FP64)
        if "stream" not in kw:
            kw["stream"] = torch.cuda.current_stream(self.device).cuda_stream
        return default_params(**kw)

    def iterate(self, y, n_iter: int, params: Params | None = None, **kw):
        """Enqueues n_iter ADMM iterations on y (CUDA tensor [L, N, N]) and returns.
        A status latched by earlier asynchronous work raises here."""
        import torch

        if params is None:
            params = self.params(**kw)
        if self.n_vis is not None:
            # visibilities: complex64 [sum M_l] (or float32 [sum M_l, 2])
            if y.dtype == torch.complex64:
                y = torch.view_as_real(y.contiguous())
            if y.dtype != torch.float32 or not y.is_cuda or tuple(y.shape) != (self.n_vis, 2):
                raise ValueError("y must be the plan's visibilities: CUDA complex64 [sum M_l]")
        elif y.dtype != self.dtype or not y.is_cuda or tuple(y.shape) != (self.L, self.N, self.N):
            raise ValueError("y must be a CUDA tensor [L, N, N] of the plan's dtype")
        y = y.contiguous()
        f = lib().mf_admm_iterate if self.dtype == torch.float32 else lib().mf_admm_iterate_f64
        _check(f(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.byref(params), int(n_iter)), "mf_admm_iterate")
        self._y_keepalive = y

    def get(self, which: int):
        import torch

        n = ctypes.c_size_t()
        _check(lib().mf_plan_get_array(self._h, which, None, ctypes.byref(n)), "mf_plan_get_array")
        out = torch.empty(n.value, dtype=self.dtype, device=self.device)
        _check(lib().mf_plan_get_array(self._h, which, ctypes.c_void_p(out.data_ptr()), ctypes.byref(n)),
               "mf_plan_get_array")
        if which == ARR_GAMMA_T:
            return out.view(-1, self.L, self.N, self.N)
        return out.view(self.L, self.N, self.N)

    def set(self, which: int, t):
        t = t.contiguous()
        _check(lib().mf_plan_set_array(self._h, which, ctypes.c_void_p(t.data_ptr()), t.numel()),
               "mf_plan_set_array")

    def x(self):
        return self.get(ARR_X)

    def report(self) -> dict:
        r = Report()
        rc = lib().mf_plan_get_report(self._h, ctypes.byref(r))
        d = r.as_dict()
        d["status"] = rc
        return d

    def set_option(self, option: int, value: int):
        """Launch-shape option (results are bitwise identical for every value)."""
        _check(lib().mf_plan_set_option(self._h, option, value), "mf_plan_set_option")

    def clear_status(self):
        """Clears a latched failure status (see mf_plan_clear_status)."""
        _check(lib().mf_plan_clear_status(self._h), "mf_plan_clear_status")

    def set_timing(self, enable: bool):
        """Per-kernel CUDA-event timing on the plan's stream (resets the counters)."""
        _check(lib().mf_plan_set_timing(self._h, int(bool(enable))), "mf_plan_set_timing")

    def timing(self) -> dict:
        """{kernel name: (total ms, launches)} since timing was last set."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            _check(lib().mf_plan_get_timing(self._h, k, ctypes.byref(ms), ctypes.byref(n)), "mf_plan_get_timing")
            out[name] = (ms.value, n.value)
        return out

    def backward(self, y, n_iter: int, dL_dX, **kw):
        """Reverse mode of n_iter unrolled iterations (tied rho): returns
        (dL/dy tensor, dL/dmu_s, dL/dmu_nu, dL/drho) for the cotangent dL_dX of
        the last X (see mf_admm_backward)."""
        import torch

        rho = kw.pop("rho", None)
        if rho is not None:
            kw.update(rho_P=rho, rho_T=rho, rho_V=rho, rho_S=rho)
        params = self.params(**kw)
        y = y.contiguous()
        g = dL_dX.contiguous()
        dy = torch.empty_like(y)
        a, b_, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().mf_admm_backward(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.byref(params), int(n_iter),
                                      ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(dy.data_ptr()),
                                      ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)), "mf_admm_backward")
        return dy, a.value, b_.value, c.value

    def get_state(self):
        import torch

        n = ctypes.c_size_t()
        _check(lib().mf_plan_get_state(self._h, None, ctypes.byref(n)), "mf_plan_get_state")
        buf = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        _check(lib().mf_plan_get_state(self._h, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(n)),
               "mf_plan_get_state")
        return buf

    def set_state(self, buf):
        _check(lib().mf_plan_set_state(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel()),
               "mf_plan_set_state")
