"""gf_eval_static: the allocation-free variant of gf_eval, for callers that
cannot allocate device memory (a plugin whose host application owns the
device heap, or a running latency-critical pipeline that may not call
cudaMalloc) and so cannot hand the library a workspace.  Its scratch is a
fixed device array inside libgf.so.

The GPU test calls it through the C ABI twice in a row and compares each
result with gf_eval (the workspace entry point) on the same inputs, within the
tolerances the other parity tests use.  This file is collected last so that a
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


@pytest.mark.gpu
def test_static_eval_matches_workspace_eval_twice(gf):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [synth.stamp64()]
    rng = np.random.default_rng(7)
    p = synth.random_params([synth.SERSIC, synth.EXPDISK, synth.SKY], rng, 70, 130)
    cases.append(synth.Stamp(70, 130, [synth.SERSIC, synth.EXPDISK, synth.SKY], p,
                             np.zeros(16, np.uint8), synth.moffat_psf(33, 3.0), os_factor=4,
                             os_box=10, name="70x130"))
    for st in cases:  # two calls in a row, different stamps
        d = gf.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
        ext = gf.model(d, st.params)
        psf = torch.as_tensor(st.psf).cuda()
        m_true = gf.convolve(d, ext, psf).cpu().numpy()
        img_h, sig_h = synth.add_noise(m_true, st.noise_seed)
        img = torch.as_tensor(img_h).cuda()
        sig = torch.as_tensor(sig_h).cuda()
        guess = st.guess()
        x_ref, m_ref = gf.evaluate(d, guess, img, sig, psf)
        model = torch.full((st.H, st.W), float("nan"), dtype=torch.float32, device="cuda")
        chi2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _static_call(gf, d, guess, img, sig, psf, model, chi2) == gf.OK, \
            gf.lib().gf_last_error()
        torch.cuda.synchronize()
        a = model.cpu().numpy().astype(np.float64)
        b = m_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(a - b) <= REL * np.abs(b) + FLOOR * np.abs(b).max())
        assert abs(chi2.item() - x_ref.item()) <= CHI2_REL * x_ref.item()
