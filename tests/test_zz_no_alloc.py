"""gf_eval_static: the allocation-free variant of gf_eval, for callers that
cannot allocate device memory (a plugin whose host application owns the
device heap, or a running latency-critical pipeline that may not call
cudaMalloc) and so cannot hand the library a workspace.  Its scratch is a
fixed device array inside libgf.so.

The GPU test calls it through the C ABI twice in a row on each of several
stamps (direct, FFT and tensor-core DFT convolution, sizes changing between
stamps) and compares each result with gf_eval (the workspace entry point) and
with the FP64 oracle on the same inputs, within the tolerances the other
parity tests use.  A CPU test pins the size limits the header documents.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1101_2254_gb300 import synth

REL, FLOOR, CHI2_REL = 1e-5, 1e-7, 1e-4


@pytest.fixture(scope="module")
def gf():
    from paper_1101_2254_gb300 import build, gf
    build.build()
    gf.lib()
    return gf


def _static_call(gf, d, params, img, sig, psf, model, chi2):
    L = gf.lib()
    p = np.ascontiguousarray(params, np.float64)
    st = L.gf_eval_static(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)),
                          C.c_void_p(img.data_ptr()), C.c_void_p(sig.data_ptr()),
                          C.c_void_p(psf.data_ptr()), C.c_void_p(model.data_ptr()),
                          C.c_void_p(chi2.data_ptr()), None)
    return st


def test_oversize_stamp_rejected_before_any_launch(gf):
    L = gf.lib()
    assert L.gf_static_scratch_bytes() == 16 << 20
    d = gf.make_desc(2048, 2048, 65, [gf.SERSIC, gf.SKY])
    p = np.zeros(9)
    st = L.gf_eval_static(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(256),
                          C.c_void_p(256), C.c_void_p(256), None, C.c_void_p(256), None)
    assert st == gf.ENOMEM
    assert b"static scratch" in L.gf_last_error()


def _eval_need(gf, H, W, P, method):
    L = gf.lib()
    L.gf_workspace_size.restype = C.c_size_t
    d = gf.make_desc(H, W, P, [gf.SERSIC, gf.SKY], conv_method=method)
    return L.gf_workspace_size(C.byref(d), None, 3)  # GF_CALL_EVAL


def test_documented_limits(gf):
    """The examples the header gives for the 16 MiB array: with a 65x65 PSF the
    default method (FFT) fits 836x836 but not 1024x1024; named direct
    convolution fits 1024x1024; a 33x33 PSF fits up to 1431x1431.  A rejected
    stamp fails with GF_ENOMEM before any launch (no device is touched)."""
    cap = 16 << 20
    assert _eval_need(gf, 836, 836, 65, gf.CONV_AUTO) <= cap
    assert _eval_need(gf, 1024, 1024, 65, gf.CONV_AUTO) > cap
    assert _eval_need(gf, 1024, 1024, 65, gf.CONV_DIRECT) <= cap
    assert _eval_need(gf, 2048, 2048, 65, gf.CONV_DIRECT) > cap
    assert _eval_need(gf, 1431, 1431, 33, gf.CONV_AUTO) <= cap
    assert _eval_need(gf, 1432, 1432, 33, gf.CONV_AUTO) > cap
    L = gf.lib()
    d = gf.make_desc(1024, 1024, 65, [gf.SERSIC, gf.SKY])
    p = np.zeros(9)
    st = L.gf_eval_static(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(256),
                          C.c_void_p(256), C.c_void_p(256), None, C.c_void_p(256), None)
    assert st == gf.ENOMEM


def _cases():
    """Stamps evaluated in this order, so that consecutive calls differ in size
    and in convolution method (direct, FFT, tensor-core DFT)."""
    rng = np.random.default_rng(7)
    out = [(synth.stamp64(), 0)]
    for H, W, P, method, osf, box in [(96, 96, 65, 0, 4, 8), (70, 130, 33, 0, 4, 10),
                                      (72, 90, 41, 3, 3, 6), (130, 70, 65, 2, 5, 8),
                                      (96, 96, 65, 3, 4, 8)]:
        kinds = [synth.SERSIC, synth.EXPDISK, synth.SKY]
        p = synth.random_params(kinds, rng, H, W)
        out.append((synth.Stamp(H, W, kinds, p, np.zeros(16, np.uint8),
                                synth.moffat_psf(P, 3.0), os_factor=osf, os_box=box,
                                name=f"{H}x{W}/P{P}"), method))
    return out


# floors of the per-pixel bound by convolution method: direct 1e-7, FFT 2e-6,
# tensor-core DFT 5e-5 of the peak (the parity tests' bounds)
_FLOOR_BY_METHOD = {0: None, 1: FLOOR, 2: 2e-6, 3: 5e-5}


@pytest.mark.gpu
def test_static_eval_matches_workspace_eval_twice(gf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    for st, method in _cases():
        d = gf.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box, conv_method=method)
        od = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
        m_true = oracle.render(od, st.params, st.psf)
        img_h, sig_h = synth.add_noise(m_true, st.noise_seed)
        img = torch.as_tensor(img_h).cuda()
        sig = torch.as_tensor(sig_h).cuda()
        psf = torch.as_tensor(st.psf).cuda()
        guess = st.guess()
        resolved = method or (2 if st.P >= 41 else 1)  # GF_AUTO_FFT_PSF
        floor = _FLOOR_BY_METHOD[resolved]
        x_ref, m_ref = gf.evaluate(d, guess, img, sig, psf)
        m_o = oracle.render(od, guess, st.psf)
        x_o = oracle.chi2(img_h, sig_h, m_o)
        b = m_ref.cpu().numpy().astype(np.float64)
        for call in range(2):  # two calls in a row on the same inputs
            model = torch.full((st.H, st.W), float("nan"), dtype=torch.float32, device="cuda")
            chi2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert _static_call(gf, d, guess, img, sig, psf, model, chi2) == gf.OK, \
                gf.lib().gf_last_error()
            torch.cuda.synchronize()
            a = model.cpu().numpy().astype(np.float64)
            # against the workspace entry point
            assert np.all(np.abs(a - b) <= REL * np.abs(b) + floor * np.abs(b).max()), \
                (st.name, method, call)
            assert abs(chi2.item() - x_ref.item()) <= CHI2_REL * x_ref.item(), (st.name, call)
            # against the FP64 oracle
            assert np.all(np.abs(a - m_o) <= REL * np.abs(m_o) + floor * np.abs(m_o).max()), \
                (st.name, method, call)
            assert abs(chi2.item() - x_o) <= CHI2_REL * x_o, (st.name, call)


def _al(x):
    return (x + 255) // 256 * 256


def _fft_len(n, even):
    m = max(n, 1)
    while True:
        if not (even and m % 2):
            r = m
            for f in (2, 3, 5):
                while r % f == 0:
                    r //= f
            if r == 1:
                return m
        m += 1


@pytest.mark.parametrize("H,W,P", [(64, 64, 33), (37, 53, 7), (128, 100, 33),  # one CTA
                                   (200, 90, 17), (64, 200, 33), (511, 512, 65)])  # three passes
def test_fft_scratch_formula(gf, H, W, P):
    """The FFT terms of the scratch formula in the header, per array rounded up
    to 256 bytes: 8 Ny (Nx/2+1) PSF spectra + 4 Ny Nx wrapped PSF + 8 (Nx + Ny)
    twiddles, and 8 He (Nx/2+1) of spectrum scratch only where the extended
    grid exceeds 160 x 160 (else Nx, Ny are padded to 96, 128 or 160 and the
    transform stays in shared memory)."""
    c = (P - 1) // 2
    He, We = H + 2 * c, W + 2 * c
    small = He <= 160 and We <= 160
    if small:
        Nx = next(32 * m for m in (3, 4, 5) if 32 * m >= We)
        Ny = next(32 * m for m in (3, 4, 5) if 32 * m >= He)
    else:
        Nx, Ny = _fft_len(We, True), _fft_len(He, False)
    Kx = Nx // 2 + 1
    extra = _al(8 * Nx) + _al(8 * Ny) + _al(8 * Ny * Kx) + _al(4 * Ny * Nx)
    extra += 0 if small else _al(8 * He * Kx)
    fft = _eval_need(gf, H, W, P, gf.CONV_FFT)
    direct = _eval_need(gf, H, W, P, gf.CONV_DIRECT)
    assert fft - direct == extra, (fft - direct, extra, small)
