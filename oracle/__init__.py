"""FP64 CPU oracle for "Fitting Galaxies on GPUs" (Barsdell, Barnes & Fluke).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of the galaxy-fitting loop (Sec. 2, steps 1-5; Sec. 3 items 1-3) in
double precision.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library: the C source lives in ``gfo.c`` and is
built by :func:`build` with gcc into ``liboracle.so`` beside it.

Every function takes and returns numpy float64 arrays; the parameter layout
per component is
    Sersic  : x0, y0, I_e, r_e, n, q, pa_deg, c
    ExpDisk : x0, y0, I_0, r_s, q, pa_deg, c
    Gaussian: x0, y0, I_0, fwhm, q, pa_deg, c
    Sky     : s0

Parity status: every function here is pinned by the tests in
``tests/test_oracle_*.py`` against closed forms, library special functions,
brute force or invariants.  The generalised-radius boxiness term (c != 0),
whose flux factor the paper does not give, is pinned by the radius on the
diagonal and by the total flux: the area of the unit superellipse, 4 Gamma(1 +
1/C)^2 / Gamma(1 + 2/C), times the elliptical closed form over pi.  The analytic
derivatives (``comp_grad``, ``model_ext_grad``, ``jacobian(analytic=True)``)
are pinned by central differences of the definitions, and db_n/dn by scipy's
inverse of the incomplete gamma and the Ciotti-Bertin expansion.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "gfo.c")
SRC_CNN = os.path.join(HERE, "gfo_cnn.c")
SRC_SPEC = os.path.join(HERE, "gfo_spec.c")

SERSIC, EXPDISK, SKY, GAUSSIAN, MOFFAT, KING, NUKER, PSF, SKYPLANE, SERSIC_F = range(1, 11)
NSLOTS = {SERSIC: 8, EXPDISK: 7, SKY: 1, GAUSSIAN: 7, MOFFAT: 8, KING: 9, NUKER: 10, PSF: 3,
          SKYPLANE: 3, SERSIC_F: 14}
CONVERGED, BADINPUT, NOCONV, MAXITER = 0, 1, 3, 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gfo.c, gfo_cnn.c and gfo_spec.c into liboracle.so with gcc
    (portable flags, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(SRC_CNN), os.path.getmtime(SRC_SPEC),
        os.path.getmtime(os.path.join(HERE, "gfo.h"))
    ):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-D_GNU_SOURCE", SRC, SRC_CNN, SRC_SPEC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class Desc(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("P", C.c_int), ("ncomp", C.c_int),
                ("kinds", C.c_int * 8), ("os_factor", C.c_int), ("os_box", C.c_int),
                ("os_x0", C.c_int), ("os_y0", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("lambda_up", C.c_double),
                ("lambda_down", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("ftol", C.c_double), ("xtol", C.c_double),
                ("fd_rel", C.c_double), ("max_iter", C.c_int), ("jac_mode", C.c_int)]


JAC_FORWARD, JAC_CENTRAL, JAC_ANALYTIC = 0, 1, 2


class Result(C.Structure):
    _fields_ = [("chi2", C.c_double), ("lam", C.c_double), ("iters", C.c_int),
                ("accepted", C.c_int), ("status", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = C.POINTER(C.c_double)
            L.gfo_bn.restype = C.c_double
            L.gfo_bn.argtypes = [C.c_double]
            L.gfo_bn_deriv.restype = C.c_double
            L.gfo_bn_deriv.argtypes = [C.c_double]
            L.gfo_comp_grad.restype = C.c_double
            L.gfo_comp_grad.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                        C.c_double, dp]
            L.gfo_model_ext_grad.restype = C.c_int
            L.gfo_model_ext_grad.argtypes = [C.POINTER(Desc), dp, C.c_int, dp]
            L.gfo_gammainc_lower.restype = C.c_double
            L.gfo_gammainc_lower.argtypes = [C.c_double, C.c_double]
            L.gfo_sersic_flux.restype = C.c_double
            L.gfo_sersic_flux.argtypes = [C.c_double] * 4
            L.gfo_moffat_alpha_per_fwhm.restype = C.c_double
            L.gfo_moffat_alpha_per_fwhm.argtypes = [C.c_double]
            L.gfo_keys_weight.restype = C.c_double
            L.gfo_keys_weight.argtypes = [C.c_double]
            L.gfo_comp_value.restype = C.c_double
            L.gfo_comp_value.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double]
            L.gfo_model_ext.restype = C.c_int
            L.gfo_model_ext.argtypes = [C.POINTER(Desc), dp, C.c_int, C.c_int, dp]
            L.gfo_convolve_direct.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
            L.gfo_convolve_fft.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp]
            L.gfo_fft.argtypes = [C.c_int, dp, dp, C.c_int]
            L.gfo_fft_size.restype = C.c_int
            L.gfo_fft_size.argtypes = [C.c_int]
            L.gfo_chi2.restype = C.c_double
            L.gfo_chi2.argtypes = [C.c_int, dp, dp, dp]
            L.gfo_eval.restype = C.c_double
            L.gfo_eval.argtypes = [C.POINTER(Desc), dp, dp, dp, dp, C.c_int, dp]
            L.gfo_jacobian.restype = C.c_double
            L.gfo_jacobian.argtypes = [C.POINTER(Desc), dp, C.c_char_p, dp, dp, dp, C.c_int,
                                       C.c_double, C.c_int, dp, dp, dp, dp]
            L.gfo_default_bounds.argtypes = [C.POINTER(Desc), dp, dp]
            L.gfo_default_opts.argtypes = [C.POINTER(Opts)]
            L.gfo_fd_step.restype = C.c_double
            L.gfo_fd_step.argtypes = [C.POINTER(Desc), C.c_int, C.c_double, C.c_double]
            L.gfo_slot_is_linear.restype = C.c_int
            L.gfo_slot_is_linear.argtypes = [C.POINTER(Desc), C.c_int]
            L.gfo_lm_fit.restype = C.c_int
            L.gfo_lm_fit.argtypes = [C.POINTER(Desc), dp, C.c_char_p, dp, dp, dp, dp, dp,
                                     C.c_int, C.POINTER(Opts), C.POINTER(Result)]
            L.gfo_lm_fit_batch.restype = C.c_int
            L.gfo_lm_fit_batch.argtypes = [C.c_int, C.POINTER(Desc), dp, C.c_char_p, dp,
                                           C.POINTER(C.c_int64), dp, dp,
                                           C.POINTER(C.c_int64), C.c_int, C.POINTER(Opts),
                                           C.POINTER(Result)]
            L.gfo_num_threads.restype = C.c_int
            L.gfo_cnn_nparams.restype = C.c_long
            L.gfo_cnn_forward.argtypes = [dp, dp, C.c_int, dp, C.c_int]
            L.gfo_cnn_loss_grad.restype = C.c_double
            L.gfo_cnn_loss_grad.argtypes = [dp, dp, dp, C.c_int, dp, C.c_int]
            L.gfo_bf16_round.restype = C.c_double
            L.gfo_bf16_round.argtypes = [C.c_double]
            L.gfo_default_guess.argtypes = [dp, C.c_int, C.c_int, dp]
            L.gfo_cnn_input.argtypes = [dp, dp, C.c_int, C.c_int, dp]
            L.gfo_cnn_encode.argtypes = [dp, C.c_int, C.c_int, dp]
            L.gfo_cnn_decode.argtypes = [dp, C.c_int, C.c_int, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_desc(H, W, P, kinds, os_factor=1, os_box=0, os_x0=-1, os_y0=-1) -> Desc:
    d = Desc()
    d.H, d.W, d.P, d.ncomp = int(H), int(W), int(P), len(kinds)
    for i, k in enumerate(kinds):
        d.kinds[i] = int(k)
    d.os_factor, d.os_box, d.os_x0, d.os_y0 = int(os_factor), int(os_box), int(os_x0), int(os_y0)
    return d


def nslots(kinds) -> int:
    return sum(NSLOTS[k] for k in kinds)


def bn(n: float) -> float:
    return lib().gfo_bn(float(n))


def bn_deriv(n: float) -> float:
    return lib().gfo_bn_deriv(float(n))


def comp_grad(kind, p, x, y):
    """(value, gradient over the component's slots) at (x, y)."""
    p = _f64(p)
    bn_ = bn(p[4]) if kind == SERSIC else 0.0
    db = bn_deriv(p[4]) if kind == SERSIC else 0.0
    g = np.zeros(10)
    v = lib().gfo_comp_grad(int(kind), _dp(p), float(x), float(y), bn_, db, _dp(g))
    return v, g[:len(p)]


def model_ext_grad(desc: Desc, params, slot: int) -> np.ndarray:
    c = (desc.P - 1) // 2
    out = np.empty((desc.H + 2 * c, desc.W + 2 * c), np.float64)
    assert lib().gfo_model_ext_grad(C.byref(desc), _dp(_f64(params)), int(slot), _dp(out)) == 0
    return out


def gammainc_lower(a: float, x: float) -> float:
    return lib().gfo_gammainc_lower(float(a), float(x))


def sersic_flux(Ie, re, n, q) -> float:
    return lib().gfo_sersic_flux(float(Ie), float(re), float(n), float(q))


def moffat_alpha_per_fwhm(beta) -> float:
    return lib().gfo_moffat_alpha_per_fwhm(float(beta))


def keys_weight(x: float) -> float:
    return lib().gfo_keys_weight(float(x))


def comp_value(kind, p, x, y) -> float:
    p = _f64(p)
    b = bn(p[4]) if kind in (SERSIC, SERSIC_F) else 0.0
    return lib().gfo_comp_value(int(kind), _dp(p), float(x), float(y), b)


def model_ext(desc: Desc, params, comp: int = -1, unit_amp: bool = False) -> np.ndarray:
    c = (desc.P - 1) // 2
    out = np.empty((desc.H + 2 * c, desc.W + 2 * c), np.float64)
    p = _f64(params)
    rc = lib().gfo_model_ext(C.byref(desc), _dp(p), int(comp), int(unit_amp), _dp(out))
    if rc != 0:
        raise ValueError("bad component kind")
    return out


def convolve_direct(ext, psf) -> np.ndarray:
    ext, psf = _f64(ext), _f64(psf)
    P = psf.shape[0]
    H, W = ext.shape[0] - (P - 1), ext.shape[1] - (P - 1)
    out = np.empty((H, W), np.float64)
    lib().gfo_convolve_direct(H, W, P, _dp(ext), _dp(psf), _dp(out))
    return out


def convolve_fft(ext, psf) -> np.ndarray:
    ext, psf = _f64(ext), _f64(psf)
    P = psf.shape[0]
    H, W = ext.shape[0] - (P - 1), ext.shape[1] - (P - 1)
    out = np.empty((H, W), np.float64)
    lib().gfo_convolve_fft(H, W, P, _dp(ext), _dp(psf), _dp(out))
    return out


def fft(x, sign=-1) -> np.ndarray:
    x = np.asarray(x, np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    lib().gfo_fft(len(x), _dp(re), _dp(im), int(sign))
    return re + 1j * im


def fft_size(n: int) -> int:
    return lib().gfo_fft_size(int(n))


def chi2(d, sigma, m) -> float:
    d, sigma, m = _f64(d), _f64(sigma), _f64(m)
    return lib().gfo_chi2(d.size, _dp(d), _dp(sigma), _dp(m))


def render(desc: Desc, params, psf, method: int = 0) -> np.ndarray:
    """Steps 1-2: the convolved model on the stamp."""
    out = np.empty((desc.H, desc.W), np.float64)
    p, psf = _f64(params), _f64(psf)
    lib().gfo_eval(C.byref(desc), _dp(p), _dp(psf), None, None, int(method), _dp(out))
    return out


def evaluate(desc: Desc, params, psf, img, sigma, method: int = 0):
    """Steps 1-3: (chi2, convolved model)."""
    out = np.empty((desc.H, desc.W), np.float64)
    p, psf, img, sigma = _f64(params), _f64(psf), _f64(img), _f64(sigma)
    x2 = lib().gfo_eval(C.byref(desc), _dp(p), _dp(psf), _dp(img), _dp(sigma), int(method),
                        _dp(out))
    return x2, out


def _fixed_bytes(fixed, ns):
    if fixed is None:
        return None
    f = np.ascontiguousarray(np.asarray(fixed, np.uint8).reshape(-1))
    assert f.size % ns == 0
    return f.tobytes()


def jacobian(desc: Desc, params, fixed, psf, img, sigma, method=0, fd_rel=1e-3,
             central=False, analytic=False):
    """Returns dict(J [nfree,H,W], A, g, chi2, model)."""
    ns = nslots([desc.kinds[i] for i in range(desc.ncomp)])
    fb = _fixed_bytes(fixed, ns)
    nfree = ns if fixed is None else int(ns - np.count_nonzero(np.asarray(fixed)))
    J = np.empty((nfree, desc.H, desc.W), np.float64)
    A = np.empty((nfree, nfree), np.float64)
    g = np.empty(nfree, np.float64)
    m = np.empty((desc.H, desc.W), np.float64)
    p, psf, img, sigma = _f64(params), _f64(psf), _f64(img), _f64(sigma)
    x2 = lib().gfo_jacobian(C.byref(desc), _dp(p), fb, _dp(psf), _dp(img), _dp(sigma),
                            int(method), float(fd_rel),
                            JAC_ANALYTIC if analytic else (JAC_CENTRAL if central else JAC_FORWARD),
                            _dp(J), _dp(A), _dp(g),
                            _dp(m))
    return dict(J=J, A=A, g=g, chi2=x2, model=m)


def default_bounds(desc: Desc):
    ns = nslots([desc.kinds[i] for i in range(desc.ncomp)])
    lo, hi = np.empty(ns), np.empty(ns)
    lib().gfo_default_bounds(C.byref(desc), _dp(lo), _dp(hi))
    return lo, hi


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().gfo_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def fd_step(desc: Desc, slot: int, v: float, fd_rel: float = 1e-3) -> float:
    return lib().gfo_fd_step(C.byref(desc), int(slot), float(v), float(fd_rel))


def slot_is_linear(desc: Desc, slot: int) -> bool:
    return bool(lib().gfo_slot_is_linear(C.byref(desc), int(slot)))


def lm_fit(desc: Desc, params, fixed, psf, img, sigma, method=0, opts: Opts | None = None,
           lo=None, hi=None):
    """Returns (params, dict(chi2, lambda, iters, accepted, status))."""
    ns = nslots([desc.kinds[i] for i in range(desc.ncomp)])
    p = np.array(params, np.float64, copy=True)
    psf, img, sigma = _f64(psf), _f64(img), _f64(sigma)
    lo, hi = _f64(lo), _f64(hi)
    r = Result()
    lib().gfo_lm_fit(C.byref(desc), _dp(p), _fixed_bytes(fixed, ns), _dp(lo), _dp(hi),
                     _dp(psf), _dp(img), _dp(sigma), int(method),
                     C.byref(opts) if opts is not None else None, C.byref(r))
    return p, dict(chi2=r.chi2, lam=r.lam, iters=r.iters, accepted=r.accepted,
                   status=r.status)


def lm_fit_batch(descs, params, fixed, psf_flat, psf_off, img_flat, sigma_flat, pix_off,
                 method=0, opts: Opts | None = None):
    """Independent fits, OpenMP across stamps.  params: [nb, nslots] (copied).
    fixed: None, one mask of nslots bytes shared by every stamp, or [nb, nslots]."""
    nb = len(descs)
    arr = (Desc * nb)(*descs)
    p = np.array(params, np.float64, copy=True)
    ns = p.shape[1]
    if fixed is not None:
        fixed = np.asarray(fixed, np.uint8).reshape(-1)
        if fixed.size == ns:
            fixed = np.tile(fixed, nb)
        if fixed.size != nb * ns:
            raise ValueError(f"fixed has {fixed.size} bytes; want {ns} or {nb * ns}")
    res = (Result * nb)()
    po = np.ascontiguousarray(psf_off, np.int64)
    xo = np.ascontiguousarray(pix_off, np.int64)
    lib().gfo_lm_fit_batch(nb, arr, _dp(p), _fixed_bytes(fixed, ns), _dp(_f64(psf_flat)),
                           po.ctypes.data_as(C.POINTER(C.c_int64)), _dp(_f64(img_flat)),
                           _dp(_f64(sigma_flat)), xo.ctypes.data_as(C.POINTER(C.c_int64)),
                           int(method), C.byref(opts) if opts is not None else None, res)
    out = [dict(chi2=r.chi2, lam=r.lam, iters=r.iters, accepted=r.accepted, status=r.status)
           for r in res]
    return p, out


def num_threads() -> int:
    return lib().gfo_num_threads()


def set_f32_emulation(on: bool) -> None:
    """Round component pixel values and convolved model pixels to float32
    (the GPU path's storage precision) from here on; off by default.  An
    experiment on the sources of GPU/oracle differences, not a mode of the
    reference computation."""
    lib().gfo_set_f32_emulation(1 if on else 0)


def set_num_threads(n: int) -> None:
    """Threads of the OpenMP loops across stamps (batched fits) from here on."""
    lib().gfo_set_num_threads(int(n))


# ---------------------------------------------------------------- spectral lines
class SpecDesc(C.Structure):
    _fields_ = [("n_chan", C.c_int), ("n_lines", C.c_int), ("n_cont", C.c_int),
                ("lsf_len", C.c_int)]


def spec_desc(n_chan, n_lines, n_cont, lsf_len) -> SpecDesc:
    return SpecDesc(int(n_chan), int(n_lines), int(n_cont), int(lsf_len))


def spec_nparams(d: SpecDesc) -> int:
    return d.n_cont + 3 * d.n_lines


def _spec_lib():
    L = lib()
    if not getattr(L, "_spec_ready", False):
        dp, sd = C.POINTER(C.c_double), C.POINTER(SpecDesc)
        L.gfo_spec_value.restype = C.c_double
        L.gfo_spec_value.argtypes = [sd, dp, C.c_double]
        L.gfo_spec_grad.restype = C.c_double
        L.gfo_spec_grad.argtypes = [sd, dp, C.c_int, C.c_double]
        L.gfo_spec_model_ext.argtypes = [sd, dp, C.c_int, dp]
        L.gfo_spec_convolve.argtypes = [sd, dp, dp, dp]
        L.gfo_spec_eval.restype = C.c_double
        L.gfo_spec_eval.argtypes = [sd, dp, dp, dp, dp, dp]
        L.gfo_spec_fd_step.restype = C.c_double
        L.gfo_spec_fd_step.argtypes = [sd, C.c_int, C.c_double, C.c_double]
        L.gfo_spec_jacobian.restype = C.c_double
        L.gfo_spec_jacobian.argtypes = [sd, dp, C.c_char_p, dp, dp, dp, C.c_int, C.c_double,
                                        dp, dp, dp]
        L.gfo_spec_default_bounds.argtypes = [sd, dp, dp]
        L.gfo_spec_fit.restype = C.c_int
        L.gfo_spec_fit.argtypes = [sd, dp, C.c_char_p, dp, dp, dp, dp, dp, C.POINTER(Opts),
                                   C.POINTER(Result)]
        L.gfo_spec_fit_batch.restype = C.c_int
        L.gfo_spec_fit_batch.argtypes = [C.c_int, sd, dp, C.c_char_p, dp, C.c_int, dp, dp,
                                         C.POINTER(Opts), C.POINTER(Result)]
        L._spec_ready = True
    return L


def spec_value(d: SpecDesc, p, x) -> float:
    return _spec_lib().gfo_spec_value(C.byref(d), _dp(_f64(p)), float(x))


def spec_grad(d: SpecDesc, p, s, x) -> float:
    return _spec_lib().gfo_spec_grad(C.byref(d), _dp(_f64(p)), int(s), float(x))


def spec_model_ext(d: SpecDesc, p, slot: int = -1) -> np.ndarray:
    E = np.zeros(d.n_chan + d.lsf_len - 1)
    _spec_lib().gfo_spec_model_ext(C.byref(d), _dp(_f64(p)), int(slot), _dp(E))
    return E


def spec_convolve(d: SpecDesc, E, lsf) -> np.ndarray:
    m = np.zeros(d.n_chan)
    _spec_lib().gfo_spec_convolve(C.byref(d), _dp(_f64(E)), _dp(_f64(lsf)), _dp(m))
    return m


def spec_eval(d: SpecDesc, p, lsf, spec=None, sig=None):
    """(chi^2, convolved model); chi^2 is 0 without data."""
    m = np.zeros(d.n_chan)
    x2 = _spec_lib().gfo_spec_eval(C.byref(d), _dp(_f64(p)), _dp(_f64(lsf)), _dp(_f64(spec)),
                                   _dp(_f64(sig)), _dp(m))
    return x2, m


def spec_fd_step(d: SpecDesc, s, v, fd_rel=1e-3) -> float:
    return _spec_lib().gfo_spec_fd_step(C.byref(d), int(s), float(v), float(fd_rel))


def spec_jacobian(d: SpecDesc, p, fixed, lsf, spec, sig, mode=JAC_FORWARD, fd_rel=1e-3):
    """dict(J [nfree, N], A, g, chi2)."""
    npar = spec_nparams(d)
    fx = _fixed_bytes(fixed, npar)
    nf = npar if fixed is None else int(npar - np.count_nonzero(np.asarray(fixed)))
    J = np.zeros((max(nf, 1), d.n_chan))
    A = np.zeros((max(nf, 1), max(nf, 1)))
    g = np.zeros(max(nf, 1))
    x2 = _spec_lib().gfo_spec_jacobian(C.byref(d), _dp(_f64(p)), fx, _dp(_f64(lsf)),
                                       _dp(_f64(spec)), _dp(_f64(sig)), int(mode), float(fd_rel),
                                       _dp(J), _dp(A), _dp(g))
    return dict(J=J[:nf], A=A[:nf, :nf], g=g[:nf], chi2=x2)


def spec_default_bounds(d: SpecDesc):
    n = spec_nparams(d)
    lo, hi = np.zeros(n), np.zeros(n)
    _spec_lib().gfo_spec_default_bounds(C.byref(d), _dp(lo), _dp(hi))
    return lo, hi


def spec_fit(d: SpecDesc, params, fixed, lsf, spec, sig, opts: Opts | None = None,
             lo=None, hi=None):
    """Returns (params, dict(chi2, lam, iters, accepted, status))."""
    p = np.array(params, np.float64, copy=True)
    r = Result()
    _spec_lib().gfo_spec_fit(C.byref(d), _dp(p), _fixed_bytes(fixed, spec_nparams(d)),
                             _dp(_f64(lo)), _dp(_f64(hi)), _dp(_f64(lsf)), _dp(_f64(spec)),
                             _dp(_f64(sig)), C.byref(opts) if opts is not None else None,
                             C.byref(r))
    return p, dict(chi2=r.chi2, lam=r.lam, iters=r.iters, accepted=r.accepted, status=r.status)


def spec_fit_batch(d: SpecDesc, params, fixed, lsf, spec, sig, opts: Opts | None = None):
    """Independent spectra (count x N), OpenMP across spectra.  lsf: L values
    shared by all, or count x L."""
    p = np.array(params, np.float64, copy=True)
    count = p.shape[0]
    lsf = _f64(lsf)
    per = int(lsf.ndim == 2)
    res = (Result * count)()
    _spec_lib().gfo_spec_fit_batch(count, C.byref(d), _dp(p), _fixed_bytes(fixed, spec_nparams(d)),
                                   _dp(lsf), per, _dp(_f64(spec)), _dp(_f64(sig)),
                                   C.byref(opts) if opts is not None else None, res)
    return p, [dict(chi2=r.chi2, lam=r.lam, iters=r.iters, accepted=r.accepted, status=r.status)
               for r in res]


# ---------------------------------------------------------------- network
def cnn_nparams() -> int:
    return int(lib().gfo_cnn_nparams())


def cnn_forward(w, x, bf16_act: bool = False) -> np.ndarray:
    """Network outputs (nb x 8) for inputs x (nb x 64 x 64); bf16_act stores the
    convolution outputs as bfloat16 (the network's specified precision)."""
    w, x = _f64(w), _f64(x)
    nb = x.shape[0]
    y = np.empty((nb, 8), np.float64)
    lib().gfo_cnn_forward(_dp(w), _dp(x), nb, _dp(y), int(bf16_act))
    return y


def cnn_loss_grad(w, x, t, bf16_act: bool = False):
    """(mean squared error, gradient) for inputs x (nb x 64 x 64) and targets t (nb x 8)."""
    w, x, t = _f64(w), _f64(x), _f64(t)
    g = np.empty_like(w)
    loss = lib().gfo_cnn_loss_grad(_dp(w), _dp(x), _dp(t), x.shape[0], _dp(g), int(bf16_act))
    return loss, g


def bf16_round(v: float) -> float:
    """Nearest bfloat16 (ties to even) of a float64 value."""
    return float(lib().gfo_bf16_round(float(v)))


def default_guess(img) -> np.ndarray:
    """Moments-based Sersic + sky start (9 slots) for an image."""
    img = _f64(img)
    out = np.empty(9, np.float64)
    lib().gfo_default_guess(_dp(img), img.shape[0], img.shape[1], _dp(out))
    return out


def cnn_input(img, sigma) -> np.ndarray:
    """Network input asinh(img / a), a = median sigma over the outer ring."""
    img = _f64(img)
    sigma = _f64(sigma)
    x = np.empty_like(img)
    lib().gfo_cnn_input(_dp(img), _dp(sigma), img.shape[0], img.shape[1], _dp(x))
    return x


def cnn_encode(p, H, W) -> np.ndarray:
    """Eight regression targets of Sersic slots p[0:7] in an H x W stamp."""
    p = _f64(p)
    t = np.empty(8)
    lib().gfo_cnn_encode(_dp(p), H, W, _dp(t))
    return t


def cnn_decode(t, H, W) -> np.ndarray:
    """Sersic slots (8, c = 0) from eight targets; I_e NaN outside the flux domain."""
    t = _f64(t)
    p = np.empty(8)
    lib().gfo_cnn_decode(_dp(t), H, W, _dp(p))
    return p
