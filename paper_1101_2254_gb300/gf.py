"""Thin Python binding of libgf.so (the C ABI in include/gf.h).

Argument marshalling only: every step of the fitting loop runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (tensors, the
workspace) and the CUDA stream.  There is no fallback: if the library is
missing or fails to load, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgf.so")

SERSIC, EXPDISK, SKY, GAUSSIAN, MOFFAT, KING, NUKER, PSF, SKYPLANE, SERSIC_F = range(1, 11)
NSLOTS = {SERSIC: 8, EXPDISK: 7, SKY: 1, GAUSSIAN: 7, MOFFAT: 8, KING: 9, NUKER: 10, PSF: 3,
          SKYPLANE: 3, SERSIC_F: 14}
CONV_AUTO, CONV_DIRECT, CONV_FFT, CONV_DFT_TC = 0, 1, 2, 3
CALL_MODEL, CALL_CONVOLVE, CALL_CHI2, CALL_EVAL, CALL_JACOBIAN, CALL_LM_FIT = range(6)
OK, EINVAL, ECUDA, ENOCONV, ESINGULAR, ENONFINITE, ETIMEOUT, ENOMEM, EMAXITER = range(9)
MAX_COMP = 8


class GFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gf status {status}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("psf_size", C.c_int), ("ncomp", C.c_int),
                ("kinds", C.c_int * MAX_COMP), ("os_factor", C.c_int), ("os_box", C.c_int),
                ("os_x0", C.c_int), ("os_y0", C.c_int), ("conv_method", C.c_int)]


class LMOpts(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("lambda_up", C.c_double),
                ("lambda_down", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("ftol", C.c_double), ("xtol", C.c_double),
                ("fd_rel", C.c_double), ("max_iter", C.c_int), ("jac_mode", C.c_int),
                ("ladder", C.c_int), ("time_budget_s", C.c_double)]


JAC_FD, JAC_ANALYTIC = 0, 1


class LMResult(C.Structure):
    _fields_ = [("chi2", C.c_double), ("lam", C.c_double), ("iters", C.c_int),
                ("accepted", C.c_int), ("status", C.c_int)]


class SpecDesc(C.Structure):
    _fields_ = [("n_chan", C.c_int), ("n_lines", C.c_int), ("n_cont", C.c_int),
                ("lsf_len", C.c_int), ("lsf_per_spectrum", C.c_int)]


class Batch(C.Structure):
    _fields_ = [("count", C.c_int), ("H", C.POINTER(C.c_int)), ("W", C.POINTER(C.c_int)),
                ("pix_off", C.POINTER(C.c_int64)), ("psf_off", C.POINTER(C.c_int64))]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libgf.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1101_2254_gb300.build`")
            L = C.CDLL(LIB_PATH)
            vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.c_void_p
            pd = C.POINTER(Desc)
            L.gf_version.restype = C.c_int
            L.gf_last_error.restype = C.c_char_p
            L.gf_nslots.restype = C.c_int
            L.gf_nslots.argtypes = [pd]
            L.gf_workspace_size.restype = C.c_size_t
            L.gf_workspace_size.argtypes = [pd, C.c_char_p, C.c_int]
            L.gf_workspace_size_batch.restype = C.c_size_t
            L.gf_workspace_size_batch.argtypes = [pd, C.POINTER(Batch), C.c_char_p]
            L.gf_default_opts.argtypes = [C.POINTER(LMOpts)]
            L.gf_model.restype = C.c_int
            L.gf_model.argtypes = [pd, dp, fp, vp, C.c_size_t, vp]
            L.gf_convolve.restype = C.c_int
            L.gf_convolve.argtypes = [pd, fp, fp, fp, vp, C.c_size_t, vp]
            L.gf_chi2.restype = C.c_int
            L.gf_chi2.argtypes = [pd, fp, fp, fp, vp, vp, C.c_size_t, vp]
            L.gf_eval.restype = C.c_int
            L.gf_eval.argtypes = [pd, dp, fp, fp, fp, fp, vp, vp, C.c_size_t, vp]
            L.gf_jacobian.restype = C.c_int
            L.gf_jacobian.argtypes = [pd, dp, C.c_char_p, C.c_double, fp, fp, fp, fp, vp, vp,
                                      vp, vp, C.c_size_t, vp]
            L.gf_jacobian_analytic.restype = C.c_int
            L.gf_jacobian_analytic.argtypes = [pd, dp, C.c_char_p, fp, fp, fp, fp, vp, vp, vp, vp,
                                               C.c_size_t, vp]
            L.gf_workspace_size_multistart.restype = C.c_size_t
            L.gf_workspace_size_multistart.argtypes = [pd, C.POINTER(Batch), C.c_int, C.c_char_p]
            L.gf_lm_fit_multistart.restype = C.c_int
            L.gf_lm_fit_multistart.argtypes = [pd, C.POINTER(Batch), C.c_int, dp, C.c_char_p, fp,
                                               fp, fp, C.POINTER(LMOpts), dp,
                                               C.POINTER(LMResult), C.POINTER(C.c_int), vp,
                                               C.c_size_t, vp]
            L.gf_lm_fit.restype = C.c_int
            L.gf_lm_fit.argtypes = [pd, dp, C.c_char_p, dp, dp, fp, fp, fp,
                                    C.POINTER(LMOpts), C.POINTER(LMResult), vp, C.c_size_t, vp]
            L.gf_lm_fit_batch.restype = C.c_int
            L.gf_lm_fit_batch.argtypes = [pd, C.POINTER(Batch), dp, C.c_char_p, fp, fp, fp,
                                          C.POINTER(LMOpts), C.POINTER(LMResult), vp,
                                          C.c_size_t, vp]
            L.gf_eval_batch.restype = C.c_int
            L.gf_eval_batch.argtypes = [pd, C.POINTER(Batch), dp, fp, fp, fp, fp, vp, vp,
                                        C.c_size_t, vp]
            L.gf_workspace_size_eval_batch.restype = C.c_size_t
            L.gf_workspace_size_eval_batch.argtypes = [pd, C.POINTER(Batch)]
            L.gf_static_scratch_bytes.restype = C.c_size_t
            L.gf_eval_static.restype = C.c_int
            L.gf_eval_static.argtypes = [pd, dp, fp, fp, fp, fp, vp, vp]
            L.gf_eval_batch_dev.restype = C.c_int
            L.gf_eval_batch_dev.argtypes = [pd, C.POINTER(Batch), vp, fp, fp, fp, fp, vp, vp,
                                            C.c_size_t, vp]
            L.gf_cnn_nparams.restype = C.c_size_t
            L.gf_cnn_workspace_size.restype = C.c_size_t
            L.gf_cnn_workspace_size.argtypes = [C.c_int, C.c_int]
            L.gf_cnn_init.restype = C.c_int
            L.gf_cnn_init.argtypes = [vp, C.c_ulonglong, vp]
            L.gf_cnn_input.restype = C.c_int
            L.gf_cnn_input.argtypes = [vp, vp, C.c_int, vp, vp]
            L.gf_cnn_forward.restype = C.c_int
            L.gf_cnn_forward.argtypes = [vp, vp, C.c_int, vp, vp, C.c_size_t, vp]
            L.gf_cnn_loss_grad.restype = C.c_int
            L.gf_cnn_loss_grad.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, C.c_size_t, vp]
            L.gf_cnn_adam.restype = C.c_int
            L.gf_cnn_adam.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, vp]
            L.gf_cnn_encode.restype = C.c_int
            L.gf_cnn_encode.argtypes = [vp, C.c_int, C.c_int, vp, vp]
            L.gf_cnn_decode.restype = C.c_int
            L.gf_cnn_decode.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp]
            L.gf_train_sample.restype = C.c_int
            L.gf_train_sample.argtypes = [C.c_ulonglong, C.c_int, C.c_int, vp, vp, vp]
            L.gf_noise.restype = C.c_int
            L.gf_noise.argtypes = [vp, C.c_int64, C.c_ulonglong, C.c_float, C.c_float, vp, vp, vp]
            L.gf_philox4x32_10.restype = C.c_int
            L.gf_philox4x32_10.argtypes = [vp, vp, C.c_int, vp]
            L.gf_workspace_size_guess.restype = C.c_size_t
            L.gf_workspace_size_guess.argtypes = [C.c_int]
            L.gf_default_guess.restype = C.c_int
            L.gf_default_guess.argtypes = [C.POINTER(Batch), vp, vp, vp, C.c_size_t, vp]
            L.gf_guess_select.restype = C.c_int
            L.gf_guess_select.argtypes = [C.c_int, vp, vp, vp, vp, dp, dp, vp, vp, vp,
                                          C.c_size_t, vp]
            L.gf_autotune.restype = C.c_int
            L.gf_autotune.argtypes = [pd, C.POINTER(Batch), vp, vp, C.c_size_t, vp]
            L.gf_conv_tile_width.restype = C.c_int
            L.gf_conv_tile_width.argtypes = [C.c_int, C.c_int]
            L.gf_set_conv_tile_width.restype = C.c_int
            L.gf_set_conv_tile_width.argtypes = [C.c_int, C.c_int, C.c_int]
            ip = C.POINTER(C.c_int)
            L.gf_conv_tile_shape.argtypes = [C.c_int, C.c_int, ip, ip, ip]
            L.gf_set_conv_tile_shape.argtypes = [C.c_int, C.c_int, C.c_int]
            L.gf_launch_count.restype = C.c_longlong
            ps = C.POINTER(SpecDesc)
            L.gf_spec_nparams.restype = C.c_int
            L.gf_spec_nparams.argtypes = [ps]
            L.gf_spec_model.argtypes = [ps, C.c_int, vp, vp, vp, vp]
            L.gf_spec_eval.argtypes = [ps, C.c_int, vp, vp, vp, vp, vp, vp, vp]
            L.gf_spec_normal.argtypes = [ps, C.c_int, vp, C.c_char_p, vp, vp, vp, C.c_int,
                                         C.c_double, vp, vp, vp, vp]
            L.gf_spec_fit.argtypes = [ps, C.c_int, vp, C.c_char_p, dp, dp, vp, vp, vp,
                                      C.POINTER(LMOpts), vp, vp, vp]
            L.gf_prof_enable.argtypes = [vp]
            L.gf_fma_peak.argtypes = [C.c_int, C.c_int, vp, C.POINTER(C.c_double), vp]
            L.gf_workspace_size_model_batch.restype = C.c_size_t
            L.gf_workspace_size_model_batch.argtypes = [C.POINTER(Desc), C.POINTER(Batch)]
            L.gf_model_batch.argtypes = [C.POINTER(Desc), C.POINTER(Batch), dp, vp, vp,
                                         C.c_size_t, vp]
            L.gf_prof_times.restype = C.c_int
            L.gf_prof_times.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
            _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise GFError(status, lib().gf_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _fixed(fixed):
    if fixed is None:
        return None
    return np.ascontiguousarray(np.asarray(fixed, np.uint8).reshape(-1)).tobytes()


def _cuda_f32(t, shape=None):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda, "expected a CUDA tensor"
    assert t.dtype == torch.float32 and t.is_contiguous(), "expected contiguous float32"
    if shape is not None:
        assert t.numel() == int(np.prod(shape)), f"expected {shape} elements, got {t.shape}"
    return t


def make_desc(H, W, psf_size, kinds, os_factor=1, os_box=0, os_x0=-1, os_y0=-1,
              conv_method=CONV_AUTO) -> Desc:
    d = Desc()
    d.H, d.W, d.psf_size, d.ncomp = int(H), int(W), int(psf_size), len(kinds)
    for i, k in enumerate(kinds):
        d.kinds[i] = int(k)
    d.os_factor, d.os_box, d.os_x0, d.os_y0 = int(os_factor), int(os_box), int(os_x0), int(os_y0)
    d.conv_method = int(conv_method)
    return d


def nslots(d: Desc) -> int:
    return lib().gf_nslots(C.byref(d))


def default_opts(**kw) -> LMOpts:
    o = LMOpts()
    lib().gf_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Workspace:
    """A reusable device workspace (a torch uint8 tensor), grown on demand."""

    def __init__(self, device=None):
        self.t = None
        self.device = device

    def get(self, nbytes: int):
        import torch
        if nbytes == 0:
            raise GFError(EINVAL, lib().gf_last_error().decode() or "workspace size 0")
        if self.t is None or self.t.numel() < nbytes:
            self.t = torch.empty(int(nbytes), dtype=torch.uint8,
                                 device=self.device or "cuda")
        return C.c_void_p(self.t.data_ptr()), C.c_size_t(self.t.numel())


_default_ws = {}


def _ws(ws):
    import torch
    if ws is not None:
        return ws
    dev = torch.cuda.current_device()
    if dev not in _default_ws:
        _default_ws[dev] = Workspace(device=f"cuda:{dev}")
    return _default_ws[dev]


def model(d: Desc, params, out=None, ws=None, stream=None):
    """Step 1: the model on the extended grid ((H+2c) x (W+2c) float32)."""
    import torch
    c = (d.psf_size - 1) // 2
    shape = (d.H + 2 * c, d.W + 2 * c)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    _cuda_f32(out, shape)
    p = _f64(params)
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), None, CALL_MODEL))
    _check(lib().gf_model(C.byref(d), _dp(p), _ptr(out), w, n, _stream(stream)))
    return out


def model_batch(d: Desc, batch, params, out=None, ws=None, stream=None):
    """Step 1 for a batch: the extended grids, packed stamp after stamp (float32)."""
    import torch
    p = np.ascontiguousarray(np.asarray(params, np.float64))
    c = (d.psf_size - 1) // 2
    n = sum((batch._keep[0][i] + 2 * c) * (batch._keep[1][i] + 2 * c) for i in range(batch.count))
    if out is None:
        out = torch.empty(int(n), dtype=torch.float32, device="cuda")
    w, nb = _ws(ws).get(lib().gf_workspace_size_model_batch(C.byref(d), C.byref(batch)))
    _check(lib().gf_model_batch(C.byref(d), C.byref(batch), _dp(p), _ptr(out), w, nb,
                                _stream(stream)))
    return out


def convolve(d: Desc, ext, psf, out=None, ws=None, stream=None):
    """Step 2: H x W valid convolution of an extended grid with the PSF."""
    import torch
    c = (d.psf_size - 1) // 2
    _cuda_f32(ext, (d.H + 2 * c, d.W + 2 * c))
    _cuda_f32(psf, (d.psf_size, d.psf_size))
    if out is None:
        out = torch.empty((d.H, d.W), dtype=torch.float32, device="cuda")
    _cuda_f32(out, (d.H, d.W))
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), None, CALL_CONVOLVE))
    _check(lib().gf_convolve(C.byref(d), _ptr(ext), _ptr(psf), _ptr(out), w, n, _stream(stream)))
    return out


def chi2(d: Desc, model_t, img, sig, out=None, ws=None, stream=None):
    """Step 3: chi^2 (float64 device scalar tensor)."""
    import torch
    for t in (model_t, img, sig):
        _cuda_f32(t, (d.H, d.W))
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), None, CALL_CHI2))
    _check(lib().gf_chi2(C.byref(d), _ptr(model_t), _ptr(img), _ptr(sig), _ptr(out), w, n,
                         _stream(stream)))
    return out


def evaluate(d: Desc, params, img, sig, psf, want_model=True, ws=None, stream=None):
    """Steps 1-3: (chi2 device tensor, convolved model or None)."""
    import torch
    for t in (img, sig):
        _cuda_f32(t, (d.H, d.W))
    _cuda_f32(psf, (d.psf_size, d.psf_size))
    m = torch.empty((d.H, d.W), dtype=torch.float32, device="cuda") if want_model else None
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    p = _f64(params)
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), None, CALL_EVAL))
    _check(lib().gf_eval(C.byref(d), _dp(p), _ptr(img), _ptr(sig), _ptr(psf), _ptr(m),
                         _ptr(out), w, n, _stream(stream)))
    return out, m


def jacobian(d: Desc, params, fixed, img, sig, psf, fd_rel=1e-3, want_J=True, ws=None,
             stream=None, analytic=False):
    """Jacobian columns and normal equations: dict(J, A, g, chi2) of device tensors.
    analytic=True: the nonlinear columns from the analytic derivatives
    (gf_jacobian_analytic) instead of forward differences."""
    import torch
    for t in (img, sig):
        _cuda_f32(t, (d.H, d.W))
    _cuda_f32(psf, (d.psf_size, d.psf_size))
    ns = nslots(d)
    fx = np.zeros(ns, np.uint8) if fixed is None else np.asarray(fixed, np.uint8)
    nf = int(ns - np.count_nonzero(fx))
    J = torch.empty((nf, d.H, d.W), dtype=torch.float32, device="cuda") if want_J else None
    A = torch.empty((nf, nf), dtype=torch.float64, device="cuda")
    g = torch.empty(nf, dtype=torch.float64, device="cuda")
    x2 = torch.empty(1, dtype=torch.float64, device="cuda")
    p = _f64(params)
    fb = _fixed(fx)
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), fb, CALL_JACOBIAN))
    if analytic:
        _check(lib().gf_jacobian_analytic(C.byref(d), _dp(p), fb, _ptr(img), _ptr(sig),
                                          _ptr(psf), _ptr(J), _ptr(A), _ptr(g), _ptr(x2), w, n,
                                          _stream(stream)))
    else:
        _check(lib().gf_jacobian(C.byref(d), _dp(p), fb, float(fd_rel), _ptr(img), _ptr(sig),
                                 _ptr(psf), _ptr(J), _ptr(A), _ptr(g), _ptr(x2), w, n,
                                 _stream(stream)))
    return dict(J=J, A=A, g=g, chi2=x2)


def _res(r: LMResult):
    return dict(chi2=r.chi2, lam=r.lam, iters=r.iters, accepted=r.accepted, status=r.status)


class Results:
    """Per-stamp results of a batched fit, over the library's result array without
    a per-stamp conversion when the call returns: item i is stamp i's result dict
    (built when read), and each field is a NumPy view (results.status, .iters,
    .accepted, .chi2, .lam)."""

    def __init__(self, arr):
        self._arr = arr
        self._np = np.ctypeslib.as_array(arr)  # structured view of the same memory

    def __len__(self):
        return len(self._arr)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [_res(self._arr[k]) for k in range(*i.indices(len(self._arr)))]
        return _res(self._arr[i])

    def __iter__(self):
        return (_res(r) for r in self._arr)

    def __getattr__(self, name):
        if name in ("chi2", "lam", "iters", "accepted", "status"):
            return self._np[name]
        raise AttributeError(name)


def lm_fit(d: Desc, params, fixed, img, sig, psf, opts: LMOpts | None = None, lo=None, hi=None,
           ws=None, stream=None):
    """Steps 1-5 for one stamp: (params, result dict).  Synchronises the stream."""
    for t in (img, sig):
        _cuda_f32(t, (d.H, d.W))
    _cuda_f32(psf, (d.psf_size, d.psf_size))
    p = np.array(params, np.float64, copy=True)
    fb = _fixed(fixed)
    r = LMResult()
    w, n = _ws(ws).get(lib().gf_workspace_size(C.byref(d), fb, CALL_LM_FIT))
    _check(lib().gf_lm_fit(C.byref(d), _dp(p), fb, _dp(_f64(lo) if lo is not None else None),
                           _dp(_f64(hi) if hi is not None else None), _ptr(img), _ptr(sig),
                           _ptr(psf), C.byref(opts) if opts is not None else None, C.byref(r),
                           w, n, _stream(stream)))
    return p, _res(r)


def make_batch(Hs, Ws, pix_off=None, psf_off=None, psf_size=None):
    """A gf_batch over packed stamps (row-major, stamp after stamp) and PSFs."""
    Hs = np.ascontiguousarray(Hs, np.int32)
    Ws = np.ascontiguousarray(Ws, np.int32)
    if pix_off is None:
        pix_off = np.concatenate([[0], np.cumsum(Hs.astype(np.int64) * Ws)[:-1]])
    if psf_off is None:
        psf_off = np.arange(len(Hs), dtype=np.int64) * int(psf_size) ** 2
    pix_off = np.ascontiguousarray(pix_off, np.int64)
    psf_off = np.ascontiguousarray(psf_off, np.int64)
    b = Batch()
    b.count = len(Hs)
    b.H = Hs.ctypes.data_as(C.POINTER(C.c_int))
    b.W = Ws.ctypes.data_as(C.POINTER(C.c_int))
    b.pix_off = pix_off.ctypes.data_as(C.POINTER(C.c_int64))
    b.psf_off = psf_off.ctypes.data_as(C.POINTER(C.c_int64))
    b._keep = (Hs, Ws, pix_off, psf_off)
    return b


def evaluate_batch(d: Desc, batch: Batch, params, img, sig, psf, want_model=False, ws=None,
                   stream=None):
    """Steps 1-3 for a batch: (chi2 [count] float64 device tensor, packed models or None)."""
    import torch
    p = np.ascontiguousarray(np.asarray(params, np.float64))
    x2 = torch.empty(batch.count, dtype=torch.float64, device="cuda")
    m = torch.empty_like(img) if want_model else None
    w, n = _ws(ws).get(lib().gf_workspace_size_eval_batch(C.byref(d), C.byref(batch)))
    _check(lib().gf_eval_batch(C.byref(d), C.byref(batch), _dp(p), _ptr(img), _ptr(sig),
                               _ptr(psf), _ptr(m), _ptr(x2), w, n, _stream(stream)))
    return x2, m


def lm_fit_batch(d: Desc, batch: Batch, params, fixed, img, sig, psf,
                 opts: LMOpts | None = None, ws=None, stream=None):
    """Steps 1-5 for a batch of stamps: (params [count, nslots], Results: the per-stamp
    result dicts, and each field as an array)."""
    p = np.array(params, np.float64, copy=True)
    fb = _fixed(fixed)
    res = (LMResult * batch.count)()
    w, n = _ws(ws).get(lib().gf_workspace_size_batch(C.byref(d), C.byref(batch), fb))
    _check(lib().gf_lm_fit_batch(C.byref(d), C.byref(batch), _dp(p), fb, _ptr(img), _ptr(sig),
                                 _ptr(psf), C.byref(opts) if opts is not None else None, res,
                                 w, n, _stream(stream)))
    return p, Results(res)


def lm_fit_multistart(d: Desc, batch: Batch, starts, fixed, img, sig, psf,
                      opts: LMOpts | None = None, ws=None, stream=None):
    """Multi-start fits: starts is count x K x nslots; returns (params [count, nslots],
    Results (the per-stamp result dicts), best start index per stamp)."""
    st = np.ascontiguousarray(np.asarray(starts, np.float64))
    assert st.ndim == 3 and st.shape[0] == batch.count
    K = st.shape[1]
    fb = _fixed(fixed)
    p = np.empty((batch.count, st.shape[2]), np.float64)
    res = (LMResult * batch.count)()
    best = np.empty(batch.count, np.int32)
    w, n = _ws(ws).get(lib().gf_workspace_size_multistart(C.byref(d), C.byref(batch), K, fb))
    _check(lib().gf_lm_fit_multistart(C.byref(d), C.byref(batch), K, _dp(st), fb, _ptr(img),
                                      _ptr(sig), _ptr(psf),
                                      C.byref(opts) if opts is not None else None,
                                      _dp(p), res, best.ctypes.data_as(C.POINTER(C.c_int)),
                                      w, n, _stream(stream)))
    return p, Results(res), best


def evaluate_batch_dev(d: Desc, batch: Batch, params_dev, img, sig, psf, want_model=False,
                       ws=None, stream=None):
    """evaluate_batch with the parameters in a device float64 tensor (count x nslots).
    img = sig = None renders only: returns (None, packed convolved models)."""
    import torch
    assert params_dev.dtype == torch.float64 and params_dev.is_cuda
    p = params_dev.contiguous()
    render = img is None and sig is None
    x2 = None if render else torch.empty(batch.count, dtype=torch.float64, device=p.device)
    m = None
    if render or want_model:
        npix = int(sum(int(h) * int(w) for h, w in zip(batch._keep[0], batch._keep[1])))
        m = torch.empty(npix if img is None else img.numel(), dtype=torch.float32, device=p.device)
    w, n = _ws(ws).get(lib().gf_workspace_size_eval_batch(C.byref(d), C.byref(batch)))
    _check(lib().gf_eval_batch_dev(C.byref(d), C.byref(batch), _ptr(p), _ptr(img), _ptr(sig),
                                   _ptr(psf), _ptr(m), _ptr(x2), w, n, _stream(stream)))
    return x2, m


# ------------------------------------------------------ learned initial guess
CNN_SIDE, CNN_NOUT = 64, 8
GUESS_SLOTS = 9  # Sersic (8) + sky


def cnn_nparams() -> int:
    return int(lib().gf_cnn_nparams())


def cnn_init(seed: int, stream=None):
    """He-normal initial network parameters (float32 device tensor)."""
    import torch
    w = torch.empty(cnn_nparams(), dtype=torch.float32, device="cuda")
    _check(lib().gf_cnn_init(_ptr(w), seed, _stream(stream)))
    return w


def cnn_input(img, sig, stream=None):
    """asinh(img / a) per 64x64 stamp (a = median ring sigma): float32 [B, 64, 64]."""
    import torch
    B = img.numel() // (CNN_SIDE * CNN_SIDE)
    x = torch.empty(B, CNN_SIDE, CNN_SIDE, dtype=torch.float32, device=img.device)
    _check(lib().gf_cnn_input(_ptr(img), _ptr(sig), B, _ptr(x), _stream(stream)))
    return x


def cnn_forward(w, x, ws=None, stream=None):
    """Network outputs [B, 8] (float32) for scaled inputs x [B, 64, 64]."""
    import torch
    B = x.numel() // (CNN_SIDE * CNN_SIDE)
    y = torch.empty(B, CNN_NOUT, dtype=torch.float32, device=x.device)
    wk, n = _ws(ws).get(lib().gf_cnn_workspace_size(B, 0))
    _check(lib().gf_cnn_forward(_ptr(w), _ptr(x), B, _ptr(y), wk, n, _stream(stream)))
    return y


def cnn_loss_grad(w, x, t, ws=None, grad=None, loss=None, stream=None):
    """(loss [1], grad [nparams]) device tensors of the mean squared error."""
    import torch
    B = x.numel() // (CNN_SIDE * CNN_SIDE)
    if grad is None:
        grad = torch.empty_like(w)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
    wk, n = _ws(ws).get(lib().gf_cnn_workspace_size(B, 1))
    _check(lib().gf_cnn_loss_grad(_ptr(w), _ptr(x), _ptr(t), B, _ptr(loss), _ptr(grad), wk, n,
                                  _stream(stream)))
    return loss, grad


def cnn_adam(w, m, v, grad, step: int, lr: float, stream=None):
    _check(lib().gf_cnn_adam(_ptr(w), _ptr(m), _ptr(v), _ptr(grad), step, lr, _stream(stream)))


def cnn_encode(params_dev, stream=None):
    """Targets [count, 8] of device parameters [count, nslots] (64x64 stamps)."""
    import torch
    p = params_dev.contiguous()
    t = torch.empty(p.shape[0], CNN_NOUT, dtype=torch.float32, device=p.device)
    _check(lib().gf_cnn_encode(_ptr(p), p.shape[1], p.shape[0], _ptr(t), _stream(stream)))
    return t


DECODE_MOMENT_CENTRE = 1


def cnn_decode(y, dflt, moment_centre=False, stream=None):
    """Parameters [count, 9] from network outputs; sky (and with moment_centre
    the centre) from the default starts dflt [count, 9]."""
    import torch
    out = torch.empty(y.shape[0], GUESS_SLOTS, dtype=torch.float64, device=y.device)
    flags = DECODE_MOMENT_CENTRE if moment_centre else 0
    _check(lib().gf_cnn_decode(_ptr(y.contiguous()), _ptr(dflt.contiguous()), y.shape[0], flags,
                               _ptr(out), _stream(stream)))
    return out


def train_sample(seed: int, count: int, psf_size: int = 33, stream=None):
    """(params [count, 9] float64, psfs [count, P, P] float32) of a training batch."""
    import torch
    p = torch.empty(count, GUESS_SLOTS, dtype=torch.float64, device="cuda")
    psf = torch.empty(count, psf_size, psf_size, dtype=torch.float32, device="cuda")
    _check(lib().gf_train_sample(seed, count, psf_size, _ptr(p), _ptr(psf), _stream(stream)))
    return p, psf


def noise(model_t, seed: int, sigma_read: float = 0.01, gain: float = 1.0, stream=None):
    """(image, sigma) = model + sigma * N(0, 1), sigma^2 = sigma_read^2 + max(m, 0) / gain."""
    import torch
    img = torch.empty_like(model_t)
    sig = torch.empty_like(model_t)
    _check(lib().gf_noise(_ptr(model_t), model_t.numel(), seed, sigma_read, gain, _ptr(img),
                          _ptr(sig), _stream(stream)))
    return img, sig


def philox4x32_10(blocks_in, stream=None):
    """Philox4x32-10 of int64 tensor [n, 6] (counter 4 words, key 2 words) -> [n, 4]."""
    import torch
    a = torch.as_tensor(np.asarray(blocks_in, np.uint32).view(np.int32)).cuda()
    out = torch.empty(a.shape[0], 4, dtype=torch.int32, device="cuda")
    _check(lib().gf_philox4x32_10(_ptr(a), _ptr(out), a.shape[0], _stream(stream)))
    return out.cpu().numpy().view(np.uint32)


def default_guess(batch: Batch, img, ws=None, stream=None):
    """Moments-based single-Sersic + sky starts [count, 9] (float64 device tensor)."""
    import torch
    out = torch.empty(batch.count, GUESS_SLOTS, dtype=torch.float64, device=img.device)
    wk, n = _ws(ws).get(lib().gf_workspace_size_guess(batch.count))
    _check(lib().gf_default_guess(C.byref(batch), _ptr(img), _ptr(out), wk, n, _stream(stream)))
    return out


def guess_select(cand, x2_cand, dflt, x2_dflt, lo=None, hi=None, ws=None, stream=None):
    """(starts [count, 9], choice [count] int32: 1 where the candidate was kept)."""
    import torch
    count = cand.shape[0]
    out = torch.empty_like(dflt)
    choice = torch.empty(count, dtype=torch.int32, device=cand.device)
    wk, n = _ws(ws).get(lib().gf_workspace_size_guess(count))
    lo_a = _f64(lo) if lo is not None else None
    hi_a = _f64(hi) if hi is not None else None
    _check(lib().gf_guess_select(count, _ptr(cand.contiguous()), _ptr(x2_cand),
                                 _ptr(dflt.contiguous()), _ptr(x2_dflt), _dp(lo_a), _dp(hi_a),
                                 _ptr(out), _ptr(choice), wk, n, _stream(stream)))
    return out, choice


def autotune(d: Desc, batch: Batch, psf, ws=None, stream=None):
    """Time the direct convolution's launch shapes on the batch (tile width per
    odd width class, tile height and persistent grid) and keep the fastest on
    this device (a no-op for Fourier-space convolution)."""
    w, n = _ws(ws).get(lib().gf_workspace_size_batch(C.byref(d), C.byref(batch), None))
    _check(lib().gf_autotune(C.byref(d), C.byref(batch), _ptr(psf), w, n, _stream(stream)))


def conv_tile_width(psf_size: int, width: int) -> int:
    return int(lib().gf_conv_tile_width(psf_size, width))


def set_conv_tile_width(psf_size: int, width: int, tile_w: int):
    _check(lib().gf_set_conv_tile_width(psf_size, width, tile_w))


def conv_tile_shape(psf_size: int, width: int):
    """(tile width, tile height, CTAs per SM) of the direct convolution on the
    current device for PSF side psf_size and stamp width `width`."""
    tw, th, cap = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(lib().gf_conv_tile_shape(psf_size, width, C.byref(tw), C.byref(th), C.byref(cap)))
    return tw.value, th.value, cap.value


def set_conv_tile_shape(psf_size: int, tile_h: int, ctas_per_sm: int):
    _check(lib().gf_set_conv_tile_shape(psf_size, tile_h, ctas_per_sm))


PROF_CLASSES = ("model", "conv", "reduce", "lm")


def fma_peak(fp64: bool = False, reps: int = 20, stream=None) -> float:
    """Measured FMA peak of the current device in TFLOP/s (gf_fma_peak)."""
    import torch
    sink = torch.empty(1, dtype=torch.float64, device="cuda")
    out = C.c_double(0.0)
    _check(lib().gf_fma_peak(1 if fp64 else 0, reps, C.c_void_p(sink.data_ptr()),
                             C.byref(out), _stream(stream)))
    return float(out.value)


def launch_count() -> int:
    """Kernels launched by libgf.so since it was loaded."""
    return int(lib().gf_launch_count())


class Profiler:
    """Per-kernel-class device time (CUDA events on the launching stream) and
    algorithmic work counted by the kernels themselves, while active."""

    def __init__(self):
        import torch
        self.work = torch.zeros(len(PROF_CLASSES), dtype=torch.int64, device="cuda")

    def __enter__(self):
        self.work.zero_()
        lib().gf_prof_times(None, None)  # drop anything recorded before
        lib().gf_prof_enable(C.c_void_p(self.work.data_ptr()))
        self.launch0 = launch_count()
        return self

    def __exit__(self, *exc):
        lib().gf_prof_enable(None)
        self.launches_total = launch_count() - self.launch0
        ms = (C.c_double * len(PROF_CLASSES))()
        n = (C.c_longlong * len(PROF_CLASSES))()
        lib().gf_prof_times(ms, n)
        w = self.work.cpu().tolist()
        self.result = {k: dict(ms=ms[i], launches=n[i], work=w[i])
                       for i, k in enumerate(PROF_CLASSES)}
        return False


# ------------------------------------------------------ spectral lines, cubes
def make_spec_desc(n_chan, n_lines, n_cont, lsf_len, lsf_per_spectrum=False) -> SpecDesc:
    return SpecDesc(int(n_chan), int(n_lines), int(n_cont), int(lsf_len), int(bool(lsf_per_spectrum)))


def spec_nparams(d: SpecDesc) -> int:
    n = lib().gf_spec_nparams(C.byref(d))
    if n < 0:
        _check(EINVAL)
    return n


def _cuda_f64(t, shape):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda, "expected a CUDA tensor"
    assert t.dtype == torch.float64 and t.is_contiguous(), "expected contiguous float64"
    assert t.numel() == int(np.prod(shape)), f"expected {shape} elements, got {t.shape}"
    return t


def _spec_params(d: SpecDesc, params):
    """params as a contiguous float64 CUDA tensor of count x nparams."""
    import torch
    npar = spec_nparams(d)
    if not isinstance(params, torch.Tensor):
        params = torch.as_tensor(np.asarray(params, np.float64).reshape(-1, npar), device="cuda")
    params = params.reshape(-1, npar)
    return _cuda_f64(params.contiguous(), (params.shape[0], npar)), params.shape[0]


def _spec_lsf(d: SpecDesc, lsf, count):
    return _cuda_f32(lsf, (count if d.lsf_per_spectrum else 1, d.lsf_len))


def spec_model(d: SpecDesc, params, lsf, stream=None):
    """Convolved models (count x n_chan float32) of the spectra in params."""
    import torch
    p, count = _spec_params(d, params)
    _spec_lsf(d, lsf, count)
    out = torch.empty((count, d.n_chan), dtype=torch.float32, device=p.device)
    _check(lib().gf_spec_model(C.byref(d), count, _ptr(p), _ptr(lsf), _ptr(out), _stream(stream)))
    return out


def spec_eval(d: SpecDesc, params, spec, sig, lsf, want_model=False, stream=None):
    """(chi^2 per spectrum, model or None)."""
    import torch
    p, count = _spec_params(d, params)
    for t in (spec, sig):
        _cuda_f32(t, (count, d.n_chan))
    _spec_lsf(d, lsf, count)
    x2 = torch.empty(count, dtype=torch.float64, device=p.device)
    m = torch.empty((count, d.n_chan), dtype=torch.float32, device=p.device) if want_model else None
    _check(lib().gf_spec_eval(C.byref(d), count, _ptr(p), _ptr(spec), _ptr(sig), _ptr(lsf),
                              _ptr(x2), _ptr(m), _stream(stream)))
    return x2, m


def spec_normal(d: SpecDesc, params, fixed, spec, sig, lsf, analytic=False, fd_rel=1e-3,
                stream=None):
    """Normal equations over the free slots: dict(A [count, nf, nf], g, chi2)."""
    import torch
    p, count = _spec_params(d, params)
    for t in (spec, sig):
        _cuda_f32(t, (count, d.n_chan))
    _spec_lsf(d, lsf, count)
    npar = spec_nparams(d)
    nf = npar if fixed is None else int(npar - np.count_nonzero(np.asarray(fixed)))
    A = torch.empty((count, nf, nf), dtype=torch.float64, device=p.device)
    g = torch.empty((count, nf), dtype=torch.float64, device=p.device)
    x2 = torch.empty(count, dtype=torch.float64, device=p.device)
    _check(lib().gf_spec_normal(C.byref(d), count, _ptr(p), _fixed(fixed), _ptr(spec), _ptr(sig),
                                _ptr(lsf), JAC_ANALYTIC if analytic else JAC_FD, float(fd_rel),
                                _ptr(A), _ptr(g), _ptr(x2), _stream(stream)))
    return dict(A=A, g=g, chi2=x2)


def spec_fit(d: SpecDesc, params, fixed, spec, sig, lsf, opts: LMOpts | None = None, lo=None,
             hi=None, out=None, stream=None):
    """Batched LM over the spectra (each fitted independently): returns
    (params tensor count x nparams, result tensor) on the device; see
    spec_results for the per-spectrum dicts."""
    import torch
    p, count = _spec_params(d, params)
    for t in (spec, sig):
        _cuda_f32(t, (count, d.n_chan))
    _spec_lsf(d, lsf, count)
    out = torch.empty_like(p) if out is None else _cuda_f64(out, tuple(p.shape))
    res = torch.empty((count, C.sizeof(LMResult)), dtype=torch.uint8, device=p.device)
    _check(lib().gf_spec_fit(C.byref(d), count, _ptr(p), _fixed(fixed),
                             _dp(_f64(lo) if lo is not None else None),
                             _dp(_f64(hi) if hi is not None else None), _ptr(spec), _ptr(sig),
                             _ptr(lsf), C.byref(opts) if opts is not None else None, _ptr(out),
                             _ptr(res), _stream(stream)))
    return out, res


def spec_results(res) -> list:
    """Per-spectrum result dicts from spec_fit's result tensor (copies to the host)."""
    raw = res.cpu().numpy().tobytes()
    n = C.sizeof(LMResult)
    return [_res(LMResult.from_buffer_copy(raw[i * n:(i + 1) * n])) for i in range(len(raw) // n)]
