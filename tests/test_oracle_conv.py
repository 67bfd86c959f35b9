"""Pins of the oracle's PSF convolution (step 2, Sec. 2; FFT + transform,
Sec. 3 item 2): the definition against a library routine, the flip
convention, the delta-PSF identity, flux conservation, FFT = direct, and the
Gaussian closed form."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth


@pytest.mark.parametrize("H,W,P", [(8, 8, 3), (5, 11, 5), (16, 9, 7), (3, 3, 3), (1, 1, 1)])
def test_direct_matches_library_valid_convolution(H, W, P):
    from scipy.signal import convolve2d
    rng = np.random.default_rng(H * 100 + W * 10 + P)
    ext = rng.standard_normal((H + P - 1, W + P - 1))
    psf = rng.uniform(0.0, 1.0, (P, P))  # asymmetric: pins the kernel flip
    want = convolve2d(ext, psf, mode="valid")
    got = oracle.convolve_direct(ext, psf)
    assert got.shape == (H, W)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_flip_convention_single_tap():
    # a PSF with one off-centre tap at (v, u) shifts the image by (v - c, u - c)
    P, c = 5, 2
    ext = np.arange(12 * 14, dtype=np.float64).reshape(12, 14)
    psf = np.zeros((P, P)); psf[c + 1, c - 2] = 1.0   # dv = +1, du = -2
    out = oracle.convolve_direct(ext, psf)
    # out(i, j) = E[i + c - dv][j + c - du]
    for i in range(out.shape[0]):
        for j in range(out.shape[1]):
            assert out[i, j] == ext[i + c - 1, j + c + 2]


def test_delta_psf_is_the_valid_crop():
    rng = np.random.default_rng(3)
    P, c = 9, 4
    ext = rng.standard_normal((20 + 2 * c, 17 + 2 * c))
    psf = np.zeros((P, P)); psf[c, c] = 1.0
    assert np.array_equal(oracle.convolve_direct(ext, psf), ext[c:-c, c:-c])
    fft = oracle.convolve_fft(ext, psf)
    assert np.abs(fft - ext[c:-c, c:-c]).max() < 1e-13 * np.abs(ext).max()


@pytest.mark.parametrize("method", ["direct", "fft"])
def test_flux_conservation(method):
    # a source whose support keeps 2c from the grid border: the valid output
    # holds the whole full-mode convolution, so sum(out) = sum(ext) sum(psf)
    rng = np.random.default_rng(5)
    P, c = 7, 3
    ext = np.zeros((30, 26))
    ext[2 * c:-2 * c, 2 * c:-2 * c] = rng.uniform(0, 1, (30 - 4 * c, 26 - 4 * c))
    psf = synth.random_psf(P, 9).astype(np.float64)
    f = oracle.convolve_direct if method == "direct" else oracle.convolve_fft
    out = f(ext, psf)
    assert abs(out.sum() - ext.sum() * psf.sum()) < 1e-12 * ext.sum()


@pytest.mark.parametrize("H,W,P", [(4, 4, 3), (16, 16, 7), (13, 10, 5), (30, 31, 25), (7, 90, 9)])
def test_fft_matches_direct(H, W, P):
    rng = np.random.default_rng(H + W + P)
    ext = rng.standard_normal((H + P - 1, W + P - 1))
    psf = rng.uniform(0, 1, (P, P))
    d = oracle.convolve_direct(ext, psf)
    f = oracle.convolve_fft(ext, psf)
    assert np.abs(f - d).max() < 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 12, 49, 90, 576, 289, 1280, 97])
def test_fft_matches_library(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.abs(oracle.fft(x, -1) - np.fft.fft(x)).max() < 1e-12 * max(1.0, np.abs(x).sum())
    assert np.abs(oracle.fft(x, +1) - n * np.fft.ifft(x)).max() < 1e-12 * max(1.0, np.abs(x).sum())


def test_fft_sizes():
    assert [oracle.fft_size(n) for n in (1, 88, 90, 91, 576, 1278, 289)] == [1, 90, 90, 96, 576, 1280, 300]


def test_gaussian_closed_form():
    # Sersic n = 1/2 is a Gaussian of amplitude 2 I_e with covariance
    # R diag(re^2, q^2 re^2) R^T / (2 ln 2); convolved with a normalised
    # Gaussian PSF of width sp it is the Gaussian with covariance Sg + sp^2 I and
    # amplitude 2 I_e sqrt(det Sg / det(Sg + sp^2 I)).  Sampling at pixel
    # centres aliases at ~exp(-2 pi^2 sp^2), negligible for sp >= 1.6.
    H = W = 48
    P, c = 25, 12
    Ie, re, q, pa = 1.0, 6.0, 0.6, 35.0
    x0, y0 = 23.4, 24.2
    sp = 4.0 / (2 * math.sqrt(2 * math.log(2)))
    d = oracle.make_desc(H, W, P, [oracle.SERSIC])
    p = np.array([x0, y0, Ie, re, 0.5, q, pa, 0.0])
    psf = synth.gaussian_psf(P, 4.0).astype(np.float64)
    out = oracle.convolve_direct(oracle.model_ext(d, p), psf)
    th = math.radians(pa)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Sg = R @ np.diag([re * re, q * q * re * re]) @ R.T / (2 * math.log(2))
    St = Sg + sp * sp * np.eye(2)
    amp = 2 * Ie * math.sqrt(np.linalg.det(Sg) / np.linalg.det(St))
    Si = np.linalg.inv(St)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    dx, dy = xx - x0, yy - y0
    want = amp * np.exp(-0.5 * (Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy))
    assert np.abs(out - want).max() < 1e-6 * want.max()
