"""Pins of the spectral-line oracle (the one-dimensional loop of Sec. 5's
"flexible dimensionality": spectral line or cube fitting) against closed
forms, library routines and known answers, none of which reuse its code."""
import math

import numpy as np
import pytest

import oracle


def _desc(N=64, K=2, nc=2, L=9):
    return oracle.spec_desc(N, K, nc, L)


def test_line_sum_is_the_gaussian_integral():
    # sum over integer x of A exp(-(x - mu)^2 / 2 s^2) = A s sqrt(2 pi) up to
    # exp(-2 pi^2 s^2) (Poisson summation): pins the amplitude and the width
    d = oracle.spec_desc(400, 1, 0, 1)
    for A, mu, s in ((2.5, 200.3, 1.5), (0.7, 180.9, 4.2), (-1.1, 210.0, 9.0)):
        E = oracle.spec_model_ext(d, [A, mu, s])
        assert abs(E.sum() - A * s * math.sqrt(2 * math.pi)) < 1e-12 * abs(A) * s


def test_line_peak_and_half_width():
    d = oracle.spec_desc(100, 1, 0, 1)
    A, mu, s = 3.0, 41.25, 2.0
    p = [A, mu, s]
    assert oracle.spec_value(d, p, mu) == A
    hw = s * math.sqrt(2 * math.log(2))  # half width at half maximum
    assert abs(oracle.spec_value(d, p, mu + hw) - A / 2) < 1e-14
    assert abs(oracle.spec_value(d, p, mu - hw) - A / 2) < 1e-14


def test_continuum_coordinate():
    # t = -1 at the first channel, +1 at the last
    N = 37
    d = oracle.spec_desc(N, 0, 3, 1)
    a = [0.4, -0.3, 0.2]
    assert abs(oracle.spec_value(d, a, 0.0) - (0.4 + 0.3 + 0.2)) < 1e-15
    assert abs(oracle.spec_value(d, a, N - 1.0) - (0.4 - 0.3 + 0.2)) < 1e-15
    assert abs(oracle.spec_value(d, a, (N - 1) / 2) - 0.4) < 1e-15


def test_convolution_is_numpy_valid_convolution():
    # numpy.convolve(E, lsf, 'valid')[i] = sum_u E[i + L - 1 - u] lsf[u]: the
    # flipped-kernel sum on the channels; an asymmetric LSF pins the flip
    rng = np.random.default_rng(3)
    d = _desc(N=50, L=11)
    E = rng.standard_normal(d.n_chan + d.lsf_len - 1)
    lsf = rng.uniform(0.0, 1.0, d.lsf_len)
    assert np.allclose(oracle.spec_convolve(d, E, lsf), np.convolve(E, lsf, "valid"),
                       rtol=0, atol=1e-13)


def test_convolution_shift_direction():
    # a delta at tap u0 maps channel i to the model at x = i + c - u0
    d = oracle.spec_desc(30, 1, 0, 7)
    p = [1.0, 12.3, 1.7]
    for u0 in (0, 2, 6):
        lsf = np.zeros(7)
        lsf[u0] = 1.0
        _, m = oracle.spec_eval(d, p, lsf)
        want = [oracle.spec_value(d, p, i + 3 - u0) for i in range(30)]
        assert np.allclose(m, want, rtol=0, atol=1e-15)


def test_gaussian_line_through_gaussian_lsf():
    # sampled Gaussians with widths >= 1.5 convolve like continuous ones (to
    # ~exp(-2 pi^2 s^2)): a line of width s through a normalised LSF of width
    # sl is a Gaussian of width S = sqrt(s^2 + sl^2) and amplitude A s / S
    s, sl, A, mu = 2.2, 1.6, 1.9, 60.4
    L = 41
    u = np.arange(L) - (L - 1) / 2
    lsf = np.exp(-0.5 * (u / sl) ** 2)
    lsf /= lsf.sum()
    d = oracle.spec_desc(120, 1, 0, L)
    _, m = oracle.spec_eval(d, [A, mu, s], lsf)
    S = math.hypot(s, sl)
    x = np.arange(120)
    want = A * s / S * np.exp(-0.5 * ((x - mu) / S) ** 2)
    assert np.abs(m - want).max() < 1e-10 * A


def test_flux_conserved_by_normalised_lsf():
    rng = np.random.default_rng(5)
    L = 15
    lsf = rng.uniform(0.0, 1.0, L)
    lsf /= lsf.sum()
    d = oracle.spec_desc(200, 2, 0, L)
    p = [1.3, 80.2, 3.0, 0.6, 120.7, 5.5]
    _, m = oracle.spec_eval(d, p, lsf)
    assert abs(m.sum() - (1.3 * 3.0 + 0.6 * 5.5) * math.sqrt(2 * math.pi)) < 1e-10


@pytest.mark.parametrize("x", [10.0, 31.4, 32.0, 47.9])
def test_gradient_matches_central_differences(x):
    d = _desc(N=64, K=2, nc=3, L=1)
    p = np.array([0.3, -0.1, 0.05, 2.0, 31.0, 2.5, -0.8, 40.0, 4.0])
    for s in range(len(p)):
        # truncation h^2 f'''/6 ~ 1e-9 of the column (widths >= 2.5), rounding
        # 1e-16 |E| / h ~ 1e-12
        h = 1e-4
        pp, pm = p.copy(), p.copy()
        pp[s] += h
        pm[s] -= h
        fd = (oracle.spec_value(d, pp, x) - oracle.spec_value(d, pm, x)) / (2 * h)
        g = oracle.spec_grad(d, p, s, x)
        assert abs(g - fd) <= 1e-7 * max(abs(fd), 1e-3) + 1e-11, (s, g, fd)


def _case(seed=0, N=96, K=2, nc=2, L=9, noise=True):
    rng = np.random.default_rng(seed)
    d = oracle.spec_desc(N, K, nc, L)
    u = np.arange(L) - (L - 1) / 2
    lsf = np.exp(-0.5 * (u / 1.3) ** 2)
    lsf /= lsf.sum()
    p = [1.0, 0.2][:nc]
    for k in range(K):
        p += [rng.uniform(3.0, 8.0), (k + 1) * N / (K + 1) + rng.uniform(-3, 3),
              rng.uniform(1.5, 4.0)]
    p = np.array(p)
    _, m = oracle.spec_eval(d, p, lsf)
    sig = np.sqrt(0.05 ** 2 + np.maximum(m, 0.0) * 0.01)
    spec = m + (rng.standard_normal(N) * sig if noise else 0.0)
    return d, p, lsf, spec, sig


def test_analytic_columns_match_central_differences():
    d, p, lsf, spec, sig = _case()
    ja = oracle.spec_jacobian(d, p, None, lsf, spec, sig, mode=oracle.JAC_ANALYTIC)
    jc = oracle.spec_jacobian(d, p, None, lsf, spec, sig, mode=oracle.JAC_CENTRAL, fd_rel=1e-6)
    for f in range(ja["J"].shape[0]):
        scale = np.abs(jc["J"][f]).max()
        assert np.abs(ja["J"][f] - jc["J"][f]).max() <= 1e-7 * scale, f


def test_forward_columns_within_their_truncation():
    # forward differences carry h f''/2; the oracle's step is 1e-3
    d, p, lsf, spec, sig = _case()
    ja = oracle.spec_jacobian(d, p, None, lsf, spec, sig, mode=oracle.JAC_ANALYTIC)
    jf = oracle.spec_jacobian(d, p, None, lsf, spec, sig, mode=oracle.JAC_FORWARD)
    for f in range(ja["J"].shape[0]):
        scale = np.abs(ja["J"][f]).max()
        assert np.abs(ja["J"][f] - jf["J"][f]).max() <= 2e-3 * scale, f


def test_normal_equations_against_numpy():
    d, p, lsf, spec, sig = _case(seed=1)
    fixed = np.zeros(len(p), np.uint8)
    fixed[1] = 1  # the continuum slope held
    r = oracle.spec_jacobian(d, p, fixed, lsf, spec, sig, mode=oracle.JAC_ANALYTIC)
    J = r["J"]
    _, m = oracle.spec_eval(d, p, lsf)
    w = 1.0 / sig ** 2
    assert np.allclose(r["A"], (J * w) @ J.T, rtol=1e-12, atol=0)
    assert np.allclose(r["g"], J @ (w * (spec - m)), rtol=1e-12, atol=1e-12)
    assert abs(r["chi2"] - np.sum(w * (spec - m) ** 2)) < 1e-12 * r["chi2"]
    assert J.shape[0] == len(p) - 1


def test_lm_recovers_noiseless_parameters():
    d, p, lsf, spec, sig = _case(seed=2, noise=False)
    start = p * np.array([1.1, 0.8, 0.9, 1.0, 1.15, 1.2, 1.0, 0.85])
    start[3] += 1.2
    start[6] -= 0.9
    for mode in (oracle.JAC_FORWARD, oracle.JAC_ANALYTIC):
        pf, res = oracle.spec_fit(d, start, None, lsf, spec, sig,
                                  opts=oracle.default_opts(jac_mode=mode))
        assert res["status"] == oracle.CONVERGED
        assert res["chi2"] < 1e-12 * d.n_chan
        assert np.abs(pf - p).max() < 1e-6 * np.abs(p).max()


def test_continuum_only_fit_is_linear_least_squares():
    # no lines: the model is linear in the coefficients, so LM lands on the
    # weighted least-squares solution of the convolved basis (numpy lstsq)
    rng = np.random.default_rng(4)
    N, L = 80, 7
    d = oracle.spec_desc(N, 0, 3, L)
    lsf = rng.uniform(0.2, 1.0, L)
    spec = 1.0 + 0.1 * rng.standard_normal(N)
    sig = np.full(N, 0.1)
    B = np.stack([oracle.spec_convolve(d, oracle.spec_model_ext(d, [0, 0, 0], s), lsf)
                  for s in range(3)], axis=1)
    want = np.linalg.lstsq(B / sig[:, None], spec / sig, rcond=None)[0]
    pf, res = oracle.spec_fit(d, [0.0, 0.0, 0.0], None, lsf, spec, sig)
    assert res["status"] == oracle.CONVERGED
    assert np.abs(pf - want).max() < 1e-8


def test_noisy_fit_is_a_stationary_point():
    d, p, lsf, spec, sig = _case(seed=6)
    pf, res = oracle.spec_fit(d, p * 1.05, None, lsf, spec, sig)
    assert res["status"] == oracle.CONVERGED
    # reduced chi^2 near 1 and a vanishing Newton step at the minimum
    assert 0.6 < res["chi2"] / (d.n_chan - len(p)) < 1.5
    r = oracle.spec_jacobian(d, pf, None, lsf, spec, sig, mode=oracle.JAC_ANALYTIC)
    step = np.linalg.solve(r["A"], r["g"])
    assert np.all(np.abs(step) < 1e-4 * np.maximum(np.abs(pf), 1.0))


def test_batch_equals_single_fits():
    cases = [_case(seed=10 + i) for i in range(4)]
    d = cases[0][0]
    params = np.stack([c[1] * 1.03 for c in cases])
    spec = np.concatenate([c[3] for c in cases])
    sig = np.concatenate([c[4] for c in cases])
    pb, rb = oracle.spec_fit_batch(d, params, None, cases[0][2], spec, sig)
    for i, c in enumerate(cases):
        ps, rs = oracle.spec_fit(d, c[1] * 1.03, None, c[2], c[3], c[4])
        assert np.array_equal(ps, pb[i]) and rs["chi2"] == rb[i]["chi2"]


def test_width_bound_holds():
    d = oracle.spec_desc(40, 1, 0, 1)
    lo, hi = oracle.spec_default_bounds(d)
    assert lo[2] == 0.25 and np.isinf(lo[0]) and np.isinf(hi).all()
    # a line much narrower than a channel: the fit stops at the bound
    x = np.arange(40)
    spec = np.where(x == 20, 1.0, 0.0)
    pf, res = oracle.spec_fit(d, [0.5, 20.0, 2.0], None, [1.0], spec, np.full(40, 0.1))
    assert pf[2] >= 0.25
