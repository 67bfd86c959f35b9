"""Pins of the oracle's chi^2 (step 3), Jacobian (step 4 input) and
Levenberg-Marquardt loop (steps 4-5), Sec. 2."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth


def _desc(st):
    return oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)


@pytest.fixture(scope="module")
def s64():
    st = synth.stamp64()
    d = _desc(st)
    m_true = oracle.render(d, st.params, st.psf)
    img, sig = synth.add_noise(m_true, st.noise_seed)
    return st, d, m_true, img, sig


# -------------------------------------------------------------------- chi2
def test_chi2_zero_and_scaling(s64):
    st, d, m_true, img, sig = s64
    assert oracle.chi2(m_true, sig, m_true) == 0.0
    x1 = oracle.chi2(img, sig, m_true)
    x2 = oracle.chi2(img, 2 * sig.astype(np.float64), m_true)
    assert abs(x2 - x1 / 4) < 1e-12 * x1


def test_chi2_of_pure_noise(s64):
    # the true model against its own noisy draw: chi^2 ~ N +- sqrt(2N)
    st, d, m_true, img, sig = s64
    N = img.size
    x = oracle.chi2(img, sig, m_true)
    assert abs(x - N) < 5 * math.sqrt(2 * N)


def test_chi2_skips_invalid_pixels_and_matches_exact_sum():
    rng = np.random.default_rng(0)
    d = rng.standard_normal(1000)
    s = rng.uniform(0.5, 2, 1000)
    m = rng.standard_normal(1000)
    s[3] = 0.0; s[5] = -1.0; d[7] = np.nan; s[9] = np.inf
    ok = np.ones(1000, bool); ok[[3, 5, 7, 9]] = False
    want = math.fsum((((d - m) / s) ** 2)[ok])
    assert abs(oracle.chi2(d, s, m) - want) < 1e-14 * want


# ---------------------------------------------------------------- Jacobian
def test_jacobian_columns(s64):
    st, d, m_true, img, sig = s64
    p = st.guess()
    fwd = oracle.jacobian(d, p, st.fixed, st.psf, img, sig, fd_rel=1e-5)
    cen = oracle.jacobian(d, p, st.fixed, st.psf, img, sig, fd_rel=1e-4, central=True)
    J, Jc = fwd["J"], cen["J"]
    for f in range(J.shape[0]):
        scale = np.abs(Jc[f]).max()
        assert np.abs(J[f] - Jc[f]).max() < 1e-3 * scale
    # linear slots: the exact column equals the finite difference of the model
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    for f, s in enumerate(free):
        if not oracle.slot_is_linear(d, s):
            continue
        h = 1e-3 * max(abs(p[s]), 1e-3)
        pp = p.copy(); pp[s] += h
        fd = (oracle.render(d, pp, st.psf) - oracle.render(d, p, st.psf)) / h
        assert np.abs(fd - J[f]).max() < 1e-6 * np.abs(J[f]).max()
    # the sky column is sum(psf) everywhere
    sky_f = free.index(st.nslots - 1)
    assert np.abs(J[sky_f] - st.psf.astype(np.float64).sum()).max() < 1e-13


def test_normal_matrix_properties(s64):
    st, d, m_true, img, sig = s64
    r = oracle.jacobian(d, st.guess(), st.fixed, st.psf, img, sig)
    A, g, J = r["A"], r["g"], r["J"]
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    # g is the gradient of -chi^2/2: a small step along g lowers chi^2
    p = st.guess()
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    x0 = r["chi2"]
    step = np.linalg.solve(A, g) * 1e-3
    pp = p.copy(); pp[free] += step
    x1, _ = oracle.evaluate(d, pp, st.psf, img, sig)
    assert x1 < x0
    # and the FP64 normal matrix equals J^T W J assembled by numpy's matmul
    W = 1.0 / sig.astype(np.float64).ravel() ** 2
    Jm = J.reshape(J.shape[0], -1)
    assert np.abs(Jm @ (W[:, None] * Jm.T) - A).max() < 1e-10 * np.abs(A).max()


# ---------------------------------------------------------------------- LM
def test_lm_recovers_noiseless_parameters(s64):
    st, d, m_true, img, sig = s64
    p, res = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, m_true, sig)
    assert res["status"] == oracle.CONVERGED
    assert res["chi2"] <= 1e-10 * m_true.size
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    rel = np.abs(p[free] - st.params[free]) / np.maximum(np.abs(st.params[free]), 1.0)
    assert rel.max() < 1e-6


def test_lm_noisy_fit_is_a_minimum(s64):
    st, d, m_true, img, sig = s64
    p, res = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, img, sig)
    assert res["status"] == oracle.CONVERGED
    N = img.size
    nfree = st.nfree
    # reduced chi^2 of a good fit to Gaussian noise
    assert abs(res["chi2"] / (N - nfree) - 1.0) < 5 * math.sqrt(2.0 / N)
    # the fit beats the true parameters and sits at a stationary point
    x_true, _ = oracle.evaluate(d, st.params, st.psf, img, sig)
    assert res["chi2"] <= x_true
    r = oracle.jacobian(d, p, st.fixed, st.psf, img, sig)
    step = np.linalg.solve(r["A"], r["g"])
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    assert np.all(np.abs(step) < 1e-4 * np.maximum(np.abs(p[free]), 1.0))


def test_lm_linear_only_is_least_squares(s64):
    # with only the amplitude and the sky free the model is linear: LM lands on
    # the weighted linear least-squares solution
    st, d, m_true, img, sig = s64
    fixed = np.ones(st.nslots, np.uint8)
    fixed[2] = 0; fixed[8] = 0
    p0 = st.params.copy(); p0[2] *= 1.3; p0[8] *= 0.5
    p, res = oracle.lm_fit(d, p0, fixed, st.psf, img, sig)
    assert res["status"] == oracle.CONVERGED
    r = oracle.jacobian(d, p0, fixed, st.psf, img, sig)
    J = r["J"].reshape(2, -1).T
    w = 1.0 / sig.astype(np.float64).ravel()
    y = img.astype(np.float64).ravel()
    sol, *_ = np.linalg.lstsq(J * w[:, None], y * w, rcond=None)
    assert abs(p[2] - sol[0]) < 1e-8 * abs(sol[0])
    assert abs(p[8] - sol[1]) < 1e-8 * abs(sol[1])


def test_lm_bad_input():
    st = synth.stamp64()
    d = _desc(st)
    fixed = np.ones(st.nslots, np.uint8)
    img = np.zeros((64, 64), np.float32)
    p, res = oracle.lm_fit(d, st.params, fixed, st.psf, img, img + 1)
    assert res["status"] == oracle.BADINPUT


def test_lm_batch_equals_single_fits():
    # the batched oracle fits each stamp on its own: a shared fixed mask (one
    # row for every stamp) and a per-stamp mask give the single-stamp fits
    sts = [synth.stamp64(), synth.stamp64()]
    sts[1].params[6] = 75.0
    descs, imgs, sigs = [], [], []
    for st in sts:
        d = _desc(st)
        img, sig = synth.add_noise(oracle.render(d, st.params, st.psf), st.noise_seed)
        descs.append(d); imgs.append(img); sigs.append(sig)
    fixed = sts[0].fixed.copy()
    fixed[6] = 1  # hold PA: a mask that differs from the all-free default
    p0 = np.array([st.guess() for st in sts])
    singles = [oracle.lm_fit(descs[k], p0[k], fixed, sts[k].psf, imgs[k], sigs[k])
               for k in range(2)]
    args = (np.concatenate([st.psf.ravel() for st in sts]), [0, sts[0].psf.size],
            np.concatenate([i.ravel() for i in imgs]), np.concatenate([s.ravel() for s in sigs]),
            [0, imgs[0].size])
    for mask in (fixed, np.tile(fixed, (2, 1))):
        pb, rb = oracle.lm_fit_batch(descs, p0, mask, *args)
        for k in range(2):
            assert np.array_equal(pb[k], singles[k][0])
            assert rb[k]["chi2"] == singles[k][1]["chi2"]
            assert pb[k][6] == p0[k][6]
    with pytest.raises(ValueError):
        oracle.lm_fit_batch(descs, p0, fixed[:-1], *args)


def test_f32_emulation_rounds_storage_only(s64):
    """The single-precision storage experiment rounds every component pixel
    value and convolved model pixel to float32 and nothing else: off, the grid
    is the FP64 one; on, it equals that grid rounded per component."""
    st, d, m_true, img, sig = s64
    ext64 = oracle.model_ext(d, st.params)
    comps = [oracle.model_ext(d, st.params, comp=k) for k in range(len(st.kinds))]
    try:
        oracle.set_f32_emulation(True)
        ext32 = oracle.model_ext(d, st.params)
        m32 = oracle.render(d, st.params, st.psf)
    finally:
        oracle.set_f32_emulation(False)
    want = sum(c.astype(np.float32).astype(np.float64) for c in comps)
    assert np.array_equal(ext32, want)
    assert np.array_equal(m32, m32.astype(np.float32).astype(np.float64))
    assert not np.array_equal(ext32, ext64)
    assert np.array_equal(oracle.model_ext(d, st.params), ext64)
