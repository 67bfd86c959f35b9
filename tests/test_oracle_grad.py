"""Pins of the oracle's analytic Jacobian (the "analytic columns" step after
finite differences, step 4 of Sec. 2): the chain-rule derivatives of every
profile slot against central differences of the definitions, db_n/dn against
an independent library inverse and the Ciotti-Bertin expansion, the pixel and
grid derivatives (oversampled block included) against differences of the grid
model, and the LM with analytic columns against the known answer."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth


def _fd_value(kind, p, x, y, s, h):
    """Central difference of the profile value in slot s (b_n re-solved)."""
    def val(pp):
        bn = oracle.bn(pp[4]) if kind == oracle.SERSIC else 0.0
        return oracle.lib().gfo_comp_value(int(kind), oracle._dp(np.ascontiguousarray(pp)),
                                           float(x), float(y), bn)
    pp, pm = p.copy(), p.copy()
    pp[s] += h
    pm[s] -= h
    return (val(pp) - val(pm)) / (2.0 * h)


CASES = [
    (oracle.SERSIC, [10.3, -4.2, 1.3, 6.0, 4.0, 0.7, 30.0, 0.0]),
    (oracle.SERSIC, [-2.0, 3.5, 0.8, 3.0, 0.5, 0.45, 117.0, 0.0]),
    (oracle.SERSIC, [1.5, 2.5, 2.0, 9.0, 1.0, 0.9, 171.0, 0.6]),
    (oracle.SERSIC, [0.0, 0.0, 1.0, 4.0, 2.5, 0.3, 64.0, -0.5]),
    (oracle.SERSIC, [5.0, 1.0, 1.7, 12.0, 7.0, 0.55, 5.0, 1.2]),
    (oracle.EXPDISK, [3.1, -1.7, 0.9, 8.0, 0.6, 80.0, 0.0]),
    (oracle.EXPDISK, [-4.0, 2.2, 1.4, 5.0, 0.85, 140.0, -0.7]),
    (oracle.MOFFAT, [2.0, -3.0, 1.1, 4.0, 2.5, 0.6, 20.0, 0.0]),
    (oracle.MOFFAT, [-1.0, 1.5, 0.7, 7.0, 0.9, 0.8, 95.0, -0.4]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_comp_grad_matches_central_differences(case):
    kind, p = CASES[case]
    p = np.array(p, np.float64)
    rng = np.random.default_rng(case)
    pts = rng.uniform(-25.0, 25.0, (40, 2))
    eight = kind in (oracle.SERSIC, oracle.MOFFAT)  # slot 4 is n or beta
    c = p[7] if eight else p[6]
    q, pa = (p[5], p[6]) if eight else (p[4], p[5])
    th = math.radians(pa)
    for x, y in pts:
        if math.hypot(x - p[0], y - p[1]) < 0.3:
            continue  # the Sersic cusp: no derivative at the centre
        xp = (x - p[0]) * math.cos(th) + (y - p[1]) * math.sin(th)
        yq = (-(x - p[0]) * math.sin(th) + (y - p[1]) * math.cos(th)) / q
        if c != 0.0 and min(abs(xp), abs(yq)) < 1.0:
            # |x'|^(c+2) has an unbounded third derivative on the axes when
            # c < 1: there central differences, not the gradient, lose accuracy
            continue
        v, g = oracle.comp_grad(kind, p, x, y)
        for s in range(len(p)):
            h = 1e-5 * max(abs(p[s]), 1.0)
            gf = _fd_value(kind, p, x, y, s, h)
            # central differences carry O(h^2) truncation and ~1e-16/h rounding
            assert abs(g[s] - gf) <= 2e-7 * max(abs(gf), 1e-3 * abs(v)) + 1e-11, \
                (kind, s, x, y, g[s], gf)


def test_sky_gradient_is_one():
    v, g = oracle.comp_grad(oracle.SKY, np.array([0.07]), 3.0, 4.0)
    assert v == 0.07 and g[0] == 1.0


@pytest.mark.parametrize("n", [0.3, 0.5, 1.0, 2.0, 4.0, 6.5, 9.5])
def test_bn_derivative_matches_library_inverse(n):
    # an independent b_n: scipy's inverse of the regularised incomplete gamma
    from scipy.special import gammaincinv
    e = 1e-5
    ref = (gammaincinv(2.0 * (n + e), 0.5) - gammaincinv(2.0 * (n - e), 0.5)) / (2.0 * e)
    assert abs(oracle.bn_deriv(n) - ref) < 1e-7 * ref


@pytest.mark.parametrize("n", [2.0, 4.0, 8.0])
def test_bn_derivative_asymptotic_series(n):
    # d/dn of Ciotti & Bertin's expansion 2n - 1/3 + 4/(405 n) + 46/(25515 n^2),
    # within the derivative of its next term, 131/(1148175 n^3)
    d = 2.0 - 4.0 / (405 * n ** 2) - 92.0 / (25515 * n ** 3)
    bound = 3.0 * 131.0 / (1148175.0 * n ** 4)
    assert abs(oracle.bn_deriv(n) - d) < bound


def _small_stamp(moffat=False):
    kinds = [oracle.SERSIC, oracle.EXPDISK, oracle.SKY]
    p = [14.6, 12.3, 1.2, 4.0, 2.7, 0.65, 40.0, 0.3,
         14.1, 12.9, 0.4, 6.0, 0.8, 120.0, 0.0,
         0.05]
    if moffat:
        kinds = [oracle.MOFFAT] + kinds
        p = [13.2, 15.1, 0.9, 3.5, 2.2, 0.7, 75.0, -0.3] + p
    d = oracle.make_desc(27, 30, 7, kinds, os_factor=4, os_box=6)
    return d, np.array(p)


@pytest.mark.parametrize("moffat", [False, True])
def test_model_grid_gradient_matches_differences(moffat):
    # the extended grid with its oversampled block, every nonlinear slot
    d, p = _small_stamp(moffat)
    for s in range(len(p)):
        if oracle.slot_is_linear(d, s):
            continue
        h = 1e-5 * max(abs(p[s]), 1.0)
        pp, pm = p.copy(), p.copy()
        pp[s] += h
        pm[s] -= h
        fd = (oracle.model_ext(d, pp) - oracle.model_ext(d, pm)) / (2.0 * h)
        an = oracle.model_ext_grad(d, p, s)
        scale = np.abs(fd).max()
        assert scale > 0
        assert np.abs(an - fd).max() <= 1e-6 * scale, (s, np.abs(an - fd).max(), scale)


@pytest.mark.parametrize("moffat", [False, True])
def test_analytic_jacobian_columns_match_central_differences(moffat):
    d, p = _small_stamp(moffat)
    st_psf = synth.random_psf(7, 3)
    img = oracle.render(d, p, st_psf) + 0.01
    sig = np.full_like(img, 0.02)
    ja = oracle.jacobian(d, p, None, st_psf, img, sig, analytic=True)
    jc = oracle.jacobian(d, p, None, st_psf, img, sig, central=True, fd_rel=1e-5)
    for f in range(ja["J"].shape[0]):
        scale = np.abs(jc["J"][f]).max()
        assert np.abs(ja["J"][f] - jc["J"][f]).max() <= 1e-6 * scale, f
    # the normal equations follow: relative to the diagonal
    dA = np.abs(ja["A"] - jc["A"]) / np.sqrt(np.outer(np.diag(jc["A"]), np.diag(jc["A"])))
    assert dA.max() < 1e-4


def test_lm_with_analytic_columns_recovers_noiseless_parameters():
    st = synth.stamp64()
    d = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
    m_true = oracle.render(d, st.params, st.psf)
    _, sig = synth.add_noise(m_true, st.noise_seed)
    opts = oracle.default_opts(jac_mode=oracle.JAC_ANALYTIC)
    p, res = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, m_true, sig, opts=opts)
    assert res["status"] == oracle.CONVERGED
    assert res["chi2"] <= 1e-10 * m_true.size
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    rel = np.abs(p[free] - st.params[free]) / np.maximum(np.abs(st.params[free]), 1.0)
    assert rel.max() < 1e-6


def test_lm_analytic_and_fd_reach_the_same_minimum():
    st = synth.stamp64()
    d = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
    img, sig = synth.add_noise(oracle.render(d, st.params, st.psf), st.noise_seed)
    pa, ra = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, img, sig,
                           opts=oracle.default_opts(jac_mode=oracle.JAC_ANALYTIC))
    pf, rf = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, img, sig)
    assert ra["status"] == oracle.CONVERGED and rf["status"] == oracle.CONVERGED
    assert abs(ra["chi2"] - rf["chi2"]) <= 1e-7 * rf["chi2"]
    # at the minimum the analytic gradient vanishes
    r = oracle.jacobian(d, pa, st.fixed, st.psf, img, sig, analytic=True)
    step = np.linalg.solve(r["A"], r["g"])
    free = [s for s in range(st.nslots) if not st.fixed[s]]
    assert np.all(np.abs(step) < 1e-4 * np.maximum(np.abs(pa[free]), 1.0))
