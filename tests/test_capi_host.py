"""CPU-only checks of the C ABI: libgf.so builds, loads without a GPU, exports
every function include/gf.h declares, and rejects bad arguments before any
launch (no CUDA call is reached, so these run on a machine without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gf():
    from paper_1101_2254_gb300 import build, gf
    build.build()
    return gf


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "gf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(gf):
    names = declared_functions()
    assert "gf_lm_fit" in names and "gf_model" in names and len(names) >= 12
    lib = gf.lib()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", gf.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (gf_\w+)", out))
    assert set(names) <= exported


def test_version_and_slots(gf):
    assert gf.lib().gf_version() >= 100
    d = gf.make_desc(64, 64, 25, [gf.SERSIC, gf.SKY])
    assert gf.nslots(d) == 9
    d = gf.make_desc(64, 64, 25, [gf.SERSIC, gf.EXPDISK, gf.SKY])
    assert gf.nslots(d) == 16


@pytest.mark.parametrize("bad", [
    dict(psf_size=24), dict(psf_size=0), dict(kinds=[gf_k] if (gf_k := 9) else []),
    dict(kinds=[3, 3]), dict(kinds=[3]), dict(H=0), dict(os_factor=5, os_box=80),
    dict(os_factor=0), dict(conv_method=1, psf_size=129), dict(conv_method=7),
])
def test_invalid_desc_rejected_before_launch(gf, bad):
    kw = dict(H=64, W=64, psf_size=25, kinds=[1, 3], os_factor=1, os_box=0, conv_method=0)
    kw.update(bad)
    d = gf.make_desc(kw["H"], kw["W"], kw["psf_size"], kw["kinds"], kw["os_factor"],
                     kw["os_box"], conv_method=kw["conv_method"])
    L = gf.lib()
    p = np.zeros(16)
    st = L.gf_model(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(16), None, 0,
                    None)
    assert st == gf.EINVAL
    assert len(L.gf_last_error()) > 0
    assert L.gf_workspace_size(C.byref(d), None, gf.CALL_LM_FIT) == 0


def test_null_and_workspace_checks(gf):
    L = gf.lib()
    d = gf.make_desc(64, 64, 25, [1, 3])
    p = np.zeros(9)
    dp = p.ctypes.data_as(C.POINTER(C.c_double))
    assert L.gf_model(C.byref(d), dp, None, None, 0, None) == gf.EINVAL
    # workspace missing / misaligned / too small
    assert L.gf_model(C.byref(d), dp, C.c_void_p(256), None, 0, None) == gf.EINVAL
    assert L.gf_model(C.byref(d), dp, C.c_void_p(256), C.c_void_p(1000), 10**9, None) == gf.EINVAL
    assert L.gf_model(C.byref(d), dp, C.c_void_p(256), C.c_void_p(1024), 8, None) == gf.ENOMEM
    # too many free slots for the LM
    d3 = gf.make_desc(64, 64, 25, [1, 2, 2])   # 22 slots
    assert L.gf_workspace_size(C.byref(d3), None, gf.CALL_LM_FIT) == 0
    fixed = np.zeros(22, np.uint8); fixed[[7, 14, 21, 20, 19, 18]] = 1
    assert L.gf_workspace_size(C.byref(d3), fixed.tobytes(), gf.CALL_LM_FIT) > 0


def test_workspace_sizes_scale(gf):
    L = gf.lib()
    small = gf.make_desc(64, 64, 25, [1, 3])
    big = gf.make_desc(512, 512, 65, [1, 2, 3])
    fixed = np.zeros(16, np.uint8); fixed[14] = 1
    a = L.gf_workspace_size(C.byref(small), None, gf.CALL_LM_FIT)
    b = L.gf_workspace_size(C.byref(big), fixed.tobytes(), gf.CALL_LM_FIT)
    assert 0 < a < b
    # the 512x512 Jacobian pass holds 14 channel grids of 576^2 floats and 14 outputs of 512^2
    assert b > 14 * 4 * (576 * 576 + 512 * 512)


def test_tile_width_setter_validates_before_touching_the_device():
    from paper_1101_2254_gb300 import gf
    L = gf.lib()
    assert L.gf_set_conv_tile_width(33, 64, 32) == gf.EINVAL  # even class: 64 only
    assert L.gf_set_conv_tile_width(33, 70, 48) == gf.EINVAL  # no such width
    assert L.gf_set_conv_tile_width(0, 70, 32) == gf.EINVAL
    assert L.gf_set_conv_tile_shape(33, 24, 8) == gf.EINVAL  # no such height
    assert L.gf_set_conv_tile_shape(33, 16, 0) == gf.EINVAL
    assert L.gf_set_conv_tile_shape(33, 16, 33) == gf.EINVAL
    assert L.gf_set_conv_tile_shape(32, 16, 8) == gf.EINVAL  # even PSF side


def test_lm_ladder_option_validated_before_launch(gf):
    L = gf.lib()
    o = gf.default_opts()
    assert o.ladder == 0  # automatic
    d = gf.make_desc(64, 64, 25, [1, 3])
    p = np.zeros(9)
    r = gf.LMResult()
    fake = C.c_void_p(256)
    for bad in (-1, 5):
        o.ladder = bad
        st = L.gf_lm_fit(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)), None, None, None,
                         fake, fake, fake, C.byref(o), C.byref(r), fake, 1 << 30, None)
        assert st == gf.EINVAL, bad
        assert b"ladder" in L.gf_last_error()
    # the LM workspace size covers the largest ladder: GF_MAX_LADDER trial channels
    one = gf.make_desc(64, 64, 25, [1, 3])
    assert L.gf_workspace_size(C.byref(one), None, gf.CALL_LM_FIT) > \
        L.gf_workspace_size(C.byref(one), None, gf.CALL_JACOBIAN) + 4 * 4 * (88 * 88 + 64 * 64)


def test_jac_mode_validated_before_launch(gf):
    L = gf.lib()
    o = gf.default_opts()
    assert o.jac_mode == gf.JAC_FD
    d = gf.make_desc(64, 64, 25, [1, 3])
    p = np.zeros(9)
    r = gf.LMResult()
    fake = C.c_void_p(256)
    o.jac_mode = 7
    st = L.gf_lm_fit(C.byref(d), p.ctypes.data_as(C.POINTER(C.c_double)), None, None, None,
                     fake, fake, fake, C.byref(o), C.byref(r), fake, 1 << 30, None)
    assert st == gf.EINVAL and b"jac_mode" in L.gf_last_error()
    # the analytic Jacobian rejects bad arguments before any launch too
    dp = p.ctypes.data_as(C.POINTER(C.c_double))
    assert L.gf_jacobian_analytic(C.byref(d), dp, None, None, fake, fake, None, fake, fake, fake,
                                  fake, 1 << 30, None) == gf.EINVAL


def test_multistart_validated_before_launch(gf):
    L = gf.lib()
    d = gf.make_desc(1, 1, 25, [1, 3])
    b = gf.make_batch([64, 64], [64, 64], psf_size=25)
    st = np.zeros((2, 3, 9))
    out = np.zeros((2, 9))
    res = (gf.LMResult * 2)()
    fake = C.c_void_p(256)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    for starts in (0, -2):
        assert L.gf_lm_fit_multistart(C.byref(d), C.byref(b), starts, dp(st), None, fake, fake,
                                      fake, None, dp(out), res, None, fake, 1 << 30,
                                      None) == gf.EINVAL
        assert L.gf_workspace_size_multistart(C.byref(d), C.byref(b), starts, None) == 0
    # the workspace of K starts is that of the batch with every stamp K times
    bk = gf.make_batch([64] * 6, [64] * 6, psf_size=25)
    assert L.gf_workspace_size_multistart(C.byref(d), C.byref(b), 3, None) == \
        L.gf_workspace_size_batch(C.byref(d), C.byref(bk), None)


@pytest.mark.parametrize("bad", [
    dict(n_chan=0), dict(n_lines=6), dict(n_lines=-1), dict(n_cont=4),
    dict(n_lines=0, n_cont=0), dict(lsf_len=8), dict(lsf_len=131), dict(lsf_len=0),
])
def test_spectral_desc_rejected_before_launch(gf, bad):
    kw = dict(n_chan=100, n_lines=2, n_cont=2, lsf_len=9)
    kw.update(bad)
    d = gf.make_spec_desc(**kw)
    L = gf.lib()
    assert L.gf_spec_nparams(C.byref(d)) == -1
    dummy = C.c_void_p(256)  # never dereferenced: validation fails first
    st = L.gf_spec_fit(C.byref(d), 4, dummy, None, None, None, dummy, dummy, dummy, None,
                       dummy, dummy, None)
    assert st == gf.EINVAL
    assert L.gf_spec_model(C.byref(d), 4, dummy, dummy, dummy, None) == gf.EINVAL


def test_spectral_calls_validate_before_launch(gf):
    L = gf.lib()
    dummy = C.c_void_p(256)
    d = gf.make_spec_desc(100, 5, 3, 9)  # 18 parameters: two must be held
    assert L.gf_spec_nparams(C.byref(d)) == 18
    st = L.gf_spec_fit(C.byref(d), 4, dummy, None, None, None, dummy, dummy, dummy, None,
                       dummy, dummy, None)
    assert st == gf.EINVAL and b"free slots" in L.gf_last_error()
    fixed = np.zeros(18, np.uint8)
    fixed[:3] = 1
    # all held: no free slot
    st = L.gf_spec_normal(C.byref(d), 4, dummy, np.ones(18, np.uint8).tobytes(), dummy, dummy,
                          dummy, gf.JAC_FD, 1e-3, dummy, dummy, dummy, None)
    assert st == gf.EINVAL
    # a bad Jacobian mode, bounds with lo > hi, a NULL output: each rejected
    st = L.gf_spec_normal(C.byref(d), 4, dummy, fixed.tobytes(), dummy, dummy, dummy, 7, 1e-3,
                          dummy, dummy, dummy, None)
    assert st == gf.EINVAL
    lo = np.zeros(18)
    hi = np.full(18, -1.0)
    st = L.gf_spec_fit(C.byref(d), 4, dummy, fixed.tobytes(),
                       lo.ctypes.data_as(C.POINTER(C.c_double)),
                       hi.ctypes.data_as(C.POINTER(C.c_double)), dummy, dummy, dummy, None,
                       dummy, dummy, None)
    assert st == gf.EINVAL and b"lo > hi" in L.gf_last_error()
    st = L.gf_spec_fit(C.byref(d), 4, dummy, fixed.tobytes(), None, None, dummy, dummy, dummy,
                       None, dummy, None, None)
    assert st == gf.EINVAL and b"NULL" in L.gf_last_error()
    # count 0 is a no-op that touches nothing
    st = L.gf_spec_fit(C.byref(d), 0, None, fixed.tobytes(), None, None, None, None, None, None,
                       None, None, None)
    assert st == gf.OK
