"""Pins of the oracle's model evaluation (step 1 of the loop, Sec. 2; a
"transform" in Sec. 3): rotation convention, generalised radius, Sersic and
exponential-disk profiles, enclosed light, oversampling and block placement."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth

S, E, K = oracle.SERSIC, oracle.EXPDISK, oracle.SKY


def sersic(x0=10.0, y0=-3.0, Ie=1.7, re=6.0, n=2.5, q=0.55, pa=30.0, c=0.0):
    return np.array([x0, y0, Ie, re, n, q, pa, c])


def test_major_axis_direction_is_ccw_from_x():
    # a point at distance r_e along the major axis (angle PA from +x, CCW toward +y)
    p = sersic()
    th = math.radians(p[6])
    x, y = p[0] + p[3] * math.cos(th), p[1] + p[3] * math.sin(th)
    assert abs(oracle.comp_value(S, p, x, y) - p[2]) < 1e-13
    # at distance q r_e along the minor axis
    x, y = p[0] - p[5] * p[3] * math.sin(th), p[1] + p[5] * p[3] * math.cos(th)
    assert abs(oracle.comp_value(S, p, x, y) - p[2]) < 1e-13
    # the mirrored direction (clockwise) is not on the isophote
    x, y = p[0] + p[3] * math.cos(-th), p[1] + p[3] * math.sin(-th)
    assert abs(oracle.comp_value(S, p, x, y) - p[2]) > 1e-3


def test_boxiness_closed_form_on_diagonal():
    # with x' = t and y'/q = t, r = (2 t^C)^{1/C} = t 2^{1/C}, C = c + 2
    for c in (-0.7, 0.0, 0.9, 1.6):
        p = sersic(c=c, n=1.0)
        th = math.radians(p[6])
        t = 4.0
        xp, yp = t, p[5] * t
        x = p[0] + xp * math.cos(th) - yp * math.sin(th)
        y = p[1] + xp * math.sin(th) + yp * math.cos(th)
        r = t * 2.0 ** (1.0 / (c + 2.0))
        b = oracle.bn(1.0)
        want = p[2] * math.exp(-b * (r / p[3] - 1.0))
        assert abs(oracle.comp_value(S, p, x, y) - want) < 1e-13 * want
        # and on the major axis the radius is |x'| for any c
        x = p[0] + t * math.cos(th)
        y = p[1] + t * math.sin(th)
        want = p[2] * math.exp(-b * (t / p[3] - 1.0))
        assert abs(oracle.comp_value(S, p, x, y) - want) < 1e-13 * want


def test_expdisk_equals_sersic_one():
    b1 = oracle.bn(1.0)
    I0, rs = 2.3, 7.0
    pd = np.array([1.0, 2.0, I0, rs, 0.4, 77.0, 0.3])
    ps = np.array([1.0, 2.0, I0 * math.exp(-b1), b1 * rs, 1.0, 0.4, 77.0, 0.3])
    for (x, y) in [(1.0, 2.0), (5.0, -3.0), (-10.0, 14.0), (30.0, 2.5)]:
        a, b = oracle.comp_value(E, pd, x, y), oracle.comp_value(S, ps, x, y)
        assert abs(a - b) < 1e-13 * max(a, 1e-300)
    # I(r_s) = I_0 / e on the major axis
    th = math.radians(77.0)
    v = oracle.comp_value(E, pd, 1.0 + rs * math.cos(th), 2.0 + rs * math.sin(th))
    assert abs(v - I0 / math.e) < 1e-13


def _enclosed(kind, p, R, nt=96, nphi=96):
    """Light inside the generalised ellipse r <= R, integrated in the
    component's own frame: x' = rho cos(phi), y' = q rho sin(phi), with the
    substitution rho = r_e t^n that makes the Sersic integrand smooth."""
    n = p[4] if kind == S else 1.0
    q = p[5] if kind == S else p[4]
    re = p[3]
    th = math.radians(p[6] if kind == S else p[5])
    tmax = (R / re) ** (1.0 / n)
    tg, tw = np.polynomial.legendre.leggauss(nt)
    t = 0.5 * tmax * (tg + 1.0)
    wt = 0.5 * tmax * tw
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    tot = 0.0
    for ti, wi in zip(t, wt):
        rho = re * ti ** n
        drho = re * n * ti ** (n - 1.0)
        for ph in phi:
            xp, yp = rho * math.cos(ph), q * rho * math.sin(ph)
            x = p[0] + xp * math.cos(th) - yp * math.sin(th)
            y = p[1] + xp * math.sin(th) + yp * math.cos(th)
            tot += wi * (2 * math.pi / nphi) * q * rho * drho * oracle.comp_value(kind, p, x, y)
    return tot


@pytest.mark.parametrize("n", [0.5, 1.0, 2.5, 4.0])
def test_effective_radius_encloses_half_the_light(n):
    p = sersic(n=n)
    F = oracle.sersic_flux(p[2], p[3], n, p[5])
    assert abs(_enclosed(S, p, p[3]) - 0.5 * F) < 1e-9 * F
    # and a wider aperture encloses F P(2n, b (R/r_e)^{1/n})
    from scipy.special import gammainc
    R = 3.0 * p[3]
    want = F * gammainc(2 * n, oracle.bn(n) * 3.0 ** (1.0 / n))
    assert abs(_enclosed(S, p, R) - want) < 1e-9 * F


def test_pixel_grid_sums_to_closed_form_flux():
    # n = 1/2 and n = 1 decay fast enough that a 96x96 grid holds all the light;
    # 8x8 oversampling everywhere approximates the cell integrals.
    for n, tol in [(0.5, 2e-5), (1.0, 2e-4)]:
        d = oracle.make_desc(96, 96, 1, [S], os_factor=8, os_box=96)
        p = np.array([47.3, 48.1, 1.0, 5.0, n, 0.6, 30.0, 0.0])
        tot = oracle.model_ext(d, p).sum()
        F = oracle.sersic_flux(1.0, 5.0, n, 0.6)
        assert abs(tot - F) < tol * F


@pytest.mark.parametrize("c", [-0.6, 0.8, 1.5])
def test_boxy_pixel_grid_sums_to_superellipse_flux(c):
    """With boxiness c the isophotes are the superellipses |x'|^C + |y'/q|^C =
    r^C, C = c + 2, whose area is q r^2 A(C) with A(C) = 4 Gamma(1 + 1/C)^2 /
    Gamma(1 + 2/C) (A(2) = pi).  The light inside a generalised radius r then
    grows by I(r) q A(C) 2 r dr, so the total flux is the ellipse's closed form
    times A(C) / pi: no quadrature of the oracle's own, only the area of the
    unit superellipse."""
    C = c + 2.0
    A = 4.0 * math.gamma(1.0 + 1.0 / C) ** 2 / math.gamma(1.0 + 2.0 / C)
    d = oracle.make_desc(96, 96, 1, [S], os_factor=8, os_box=96)
    p = np.array([47.3, 48.1, 1.0, 5.0, 0.5, 0.6, 30.0, c])
    tot = oracle.model_ext(d, p).sum()
    F = oracle.sersic_flux(1.0, 5.0, 0.5, 0.6) * A / math.pi
    assert abs(tot - F) < 1e-7 * F, (tot, F)  # agrees to ~5e-9; A(C) / pi - 1 is 10-16 %


def test_position_angle_symmetries():
    d = oracle.make_desc(40, 40, 5, [S, K])
    p = np.array([19.5, 19.5, 1.0, 6.0, 1.5, 0.5, 20.0, 0.0, 0.05])
    m = oracle.model_ext(d, p)
    # PA and PA + 180 give the same image
    p2 = p.copy(); p2[6] += 180.0
    assert np.array_equal(oracle.model_ext(d, p2), m) or np.abs(oracle.model_ext(d, p2) - m).max() < 1e-12
    # PA -> 90 - PA is the transpose when the centre is on the diagonal (x <-> y reflection)
    p3 = p.copy(); p3[6] = 90.0 - p[6]
    assert np.abs(oracle.model_ext(d, p3) - m.T).max() < 1e-12 * m.max()
    # q = 1: no dependence on PA
    p4 = p.copy(); p4[5] = 1.0
    p5 = p4.copy(); p5[6] = 71.0
    assert np.abs(oracle.model_ext(d, p4) - oracle.model_ext(d, p5)).max() < 1e-12 * m.max()


def test_extended_grid_geometry_and_sky():
    # grid pixel (ie, je) is stamp pixel (ie - c, je - c) with centre (x=j, y=i)
    d = oracle.make_desc(20, 30, 7, [S, K])
    p = np.array([12.0, 8.0, 1.0, 3.0, 1.0, 1.0, 0.0, 0.0, 0.25])
    m = oracle.model_ext(d, p)
    assert m.shape == (26, 36)
    c = 3
    # the centre pixel holds I_e e^{b_1} + sky
    assert abs(m[8 + c, 12 + c] - (math.exp(oracle.bn(1.0)) + 0.25)) < 1e-12
    # components separately and with unit amplitude
    ms = oracle.model_ext(d, p, comp=0)
    sky = oracle.model_ext(d, p, comp=1)
    assert np.allclose(sky, 0.25, rtol=0, atol=0)
    assert np.abs(ms + sky - m).max() < 1e-14
    p2 = p.copy(); p2[2] = 3.5
    assert np.abs(oracle.model_ext(d, p2, comp=0, unit_amp=True) - ms).max() < 1e-15


def test_oversampling_converges_to_cell_integral():
    # the pixel mean of s x s midpoint samples converges to the cell integral
    # as 1/s^2 (a misplaced sample offset would leave a 1/s error)
    p = np.array([0.2, -0.1, 1.0, 1.5, 0.5, 0.8, 10.0, 0.0])
    i, j = 1, 0
    g, w = np.polynomial.legendre.leggauss(24)
    cell = 0.0
    for a, wa in zip(g, w):
        for b, wb in zip(g, w):
            cell += 0.25 * wa * wb * oracle.comp_value(S, p, j + 0.5 * b, i + 0.5 * a)
    errs = []
    for s in (4, 8, 16):
        d = oracle.make_desc(3, 3, 1, [S], os_factor=s, os_box=3, os_x0=0, os_y0=0)
        v = oracle.model_ext(d, p)[i, j]
        errs.append(abs(v - cell))
    assert errs[2] < 1e-4 * cell
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
    # s = 1 is the centre sample
    d = oracle.make_desc(3, 3, 1, [S], os_factor=1, os_box=3)
    assert oracle.model_ext(d, p)[i, j] == oracle.comp_value(S, p, j, i)


def test_oversampling_block_placement():
    # B x B block centred on the stamp: rows and columns floor((H-B)/2) .. +B-1
    d1 = oracle.make_desc(16, 20, 3, [S], os_factor=1, os_box=0)
    d5 = oracle.make_desc(16, 20, 3, [S], os_factor=5, os_box=4)
    p = np.array([9.3, 7.6, 1.0, 2.0, 2.0, 0.7, 33.0, 0.0])
    c = 1
    diff = np.abs(oracle.model_ext(d5, p) - oracle.model_ext(d1, p)) > 0
    rows, cols = np.nonzero(diff)
    assert rows.min() - c == 6 and rows.max() - c == 9
    assert cols.min() - c == 8 and cols.max() - c == 11
    # an explicit origin moves it
    d5b = oracle.make_desc(16, 20, 3, [S], os_factor=5, os_box=4, os_x0=1, os_y0=2)
    rows, cols = np.nonzero(np.abs(oracle.model_ext(d5b, p) - oracle.model_ext(d1, p)) > 0)
    assert rows.min() - c == 2 and cols.min() - c == 1


def test_stamp64_central_intensity():
    # the 64x64 workload's n = 4 component peaks at I_e e^{b_4} = 2141.47354...
    p = np.array([32.3, 31.7, 1.0, 8.0, 4.0, 0.7, 30.0, 0.0])
    assert abs(oracle.comp_value(S, p, 32.3, 31.7) - 2141.47354) < 1e-4


# ---------------------------------------------------------------- Gaussian
def _gauss_sigma(fwhm):
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def test_gaussian_is_the_sersic_half_profile():
    # a Sersic n = 1/2 profile is a Gaussian: b_1/2 = ln 2 gives
    # I_e exp(-ln 2 ((r/r_e)^2 - 1)) = 2 I_e exp(-r^2 / (2 s^2)) with
    # r_e^2 = 2 ln 2 s^2; the two formulas of the oracle must agree
    fwhm, amp = 5.3, 1.7
    s = _gauss_sigma(fwhm)
    pg = np.array([1.2, -0.7, amp, fwhm, 0.6, 33.0, 0.0])
    ps = np.array([1.2, -0.7, amp / 2.0, s * math.sqrt(2.0 * math.log(2.0)), 0.5, 0.6, 33.0, 0.0])
    rng = np.random.default_rng(0)
    for x, y in rng.uniform(-12.0, 12.0, (50, 2)):
        vg = oracle.comp_value(oracle.GAUSSIAN, pg, x, y)
        vs = oracle.comp_value(oracle.SERSIC, ps, x, y)
        assert abs(vg - vs) <= 1e-13 * max(abs(vs), 1e-300)


def test_gaussian_flux_closed_form():
    # sum of the sampled profile on a fine grid = 2 pi q I_0 s^2
    fwhm, amp, q = 4.0, 1.3, 0.7
    s = _gauss_sigma(fwhm)
    p = np.array([0.0, 0.0, amp, fwhm, q, 25.0, 0.0])
    h = 0.05
    xs = np.arange(-30.0, 30.0, h) + h / 2
    tot = sum(oracle.comp_value(oracle.GAUSSIAN, p, x, y) for x in xs[::8] for y in xs[::8])
    tot *= (8 * h) ** 2
    assert abs(tot - 2.0 * math.pi * q * amp * s * s) < 1e-6 * tot


def test_gaussian_gradient_matches_central_differences():
    p = np.array([2.1, -1.3, 0.9, 6.0, 0.55, 110.0, 0.3])
    rng = np.random.default_rng(1)
    for x, y in rng.uniform(-10.0, 10.0, (30, 2)):
        v, g = oracle.comp_grad(oracle.GAUSSIAN, p, x, y)
        for s in range(len(p)):
            h = 1e-5 * max(abs(p[s]), 1.0)
            pp, pm = p.copy(), p.copy()
            pp[s] += h
            pm[s] -= h
            fd = (oracle.comp_value(oracle.GAUSSIAN, pp, x, y) -
                  oracle.comp_value(oracle.GAUSSIAN, pm, x, y)) / (2.0 * h)
            assert abs(g[s] - fd) <= 2e-7 * max(abs(fd), 1e-3 * abs(v)) + 1e-11, (s, x, y)


# ---------------------------------------------------------------- Moffat
def test_moffat_half_maximum_at_half_fwhm():
    # the FWHM slot is what its name says: I = I_0 / 2 at r = FWHM / 2 on the
    # major axis and at q FWHM / 2 on the minor axis, for any beta
    for beta in (0.8, 1.0, 2.5, 4.765, 12.0):
        fwhm, amp, q, pa = 3.7, 2.2, 0.6, 40.0
        p = np.array([0.5, -1.0, amp, fwhm, beta, q, pa, 0.0])
        th = math.radians(pa)
        for rr, ang in ((fwhm / 2, th), (q * fwhm / 2, th + math.pi / 2)):
            x, y = 0.5 + rr * math.cos(ang), -1.0 + rr * math.sin(ang)
            assert abs(oracle.comp_value(oracle.MOFFAT, p, x, y) - amp / 2) < 1e-13
        assert oracle.comp_value(oracle.MOFFAT, p, 0.5, -1.0) == amp


def test_moffat_flux_closed_form():
    # integral over the plane of (1 + r^2/alpha^2)^(-beta) on an ellipse of
    # axis ratio q: pi q alpha^2 / (beta - 1), beta > 1
    fwhm, amp, q, beta = 3.0, 0.8, 0.75, 3.5
    al = fwhm * oracle.moffat_alpha_per_fwhm(beta)
    p = np.array([0.0, 0.0, amp, fwhm, beta, q, 70.0, 0.0])
    # polar quadrature in the component's own frame, r up to 4000 alpha
    # (the tail beyond holds (4000)^(2 - 2 beta) / (beta - 1) of the flux)
    from scipy.integrate import quad
    th = math.radians(70.0)

    def ring(r):
        # the ellipse of radius r: points (r cos t, q r sin t) in the frame
        v = oracle.comp_value(oracle.MOFFAT, p, r * math.cos(th), r * math.sin(th))
        return 2.0 * math.pi * q * r * v
    tot = quad(ring, 0.0, 4000.0 * al, limit=400, epsabs=0.0, epsrel=1e-12)[0]
    assert abs(tot - math.pi * q * amp * al * al / (beta - 1.0)) < 1e-8 * tot


def test_moffat_large_beta_is_the_gaussian():
    # (1 + r^2/alpha^2)^(-beta) with alpha^2 = FWHM^2 / (4 (2^(1/beta) - 1))
    # tends to exp(-a), a = 4 ln2 r^2 / FWHM^2, the Gaussian of the same FWHM.
    # Expanding 2^(1/beta) - 1 and ln(1 + z) to second order in 1/beta:
    #   ln(I_Moffat / I_Gauss) = (a^2 - a ln 2) / (2 beta) + O(a^3 / beta^2)
    fwhm = 4.4
    pg = np.array([0.0, 0.0, 1.0, fwhm, 0.8, 10.0, 0.0])
    for beta in (1e3, 1e5):
        pm = np.array([0.0, 0.0, 1.0, fwhm, beta, 0.8, 10.0, 0.0])
        for x, y in ((0.7, 0.2), (2.0, -1.5), (-3.0, 2.5)):
            vg = oracle.comp_value(oracle.GAUSSIAN, pg, x, y)
            vm = oracle.comp_value(oracle.MOFFAT, pm, x, y)
            a = -math.log(vg)
            first = (a * a - a * math.log(2.0)) / (2.0 * beta)
            assert abs(math.log(vm / vg) - first) <= 10.0 * (1.0 + a ** 3) / beta ** 2, \
                (beta, x, y, math.log(vm / vg), first)


def test_moffat_beta_one_closed_form():
    # beta = 1: alpha = FWHM / 2 and I = I_0 / (1 + (2 r / FWHM)^2)
    p = np.array([1.0, 2.0, 1.5, 6.0, 1.0, 1.0, 0.0, 0.0])
    for x, y in ((4.0, 2.0), (1.0, -3.0), (-2.0, 6.0)):
        r = math.hypot(x - 1.0, y - 2.0)
        assert abs(oracle.comp_value(oracle.MOFFAT, p, x, y) - 1.5 / (1.0 + (2 * r / 6.0) ** 2)) < 1e-14


@pytest.mark.parametrize("c", [0.0, 0.4])
def test_moffat_gradient_matches_central_differences(c):
    p = np.array([-1.2, 0.7, 1.4, 5.0, 2.7, 0.65, 128.0, c])
    rng = np.random.default_rng(2)
    th = math.radians(p[6])
    for x, y in rng.uniform(-10.0, 10.0, (30, 2)):
        xp = (x - p[0]) * math.cos(th) + (y - p[1]) * math.sin(th)
        yq = (-(x - p[0]) * math.sin(th) + (y - p[1]) * math.cos(th)) / p[5]
        if c != 0.0 and min(abs(xp), abs(yq)) < 1.0:
            continue  # as for the Sersic pins: differences lose accuracy on the axes
        v, g = oracle.comp_grad(oracle.MOFFAT, p, x, y)
        for s in range(len(p)):
            h = 1e-5 * max(abs(p[s]), 1.0)
            pp, pm = p.copy(), p.copy()
            pp[s] += h
            pm[s] -= h
            fd = (oracle.comp_value(oracle.MOFFAT, pp, x, y) -
                  oracle.comp_value(oracle.MOFFAT, pm, x, y)) / (2.0 * h)
            assert abs(g[s] - fd) <= 2e-7 * max(abs(fd), 1e-3 * abs(v)) + 1e-11, (s, x, y)


def test_gaussian_and_moffat_render_conserves_closed_form_flux():
    # The whole oracle render (pixel grid with an oversampled block, then the
    # convolution with a normalised PSF) holds each family's total light:
    # Gaussian 2 pi q I_0 s^2, Moffat pi q I_0 alpha^2 / (beta - 1).  The
    # stamp is wide enough for the Gaussian's tail; the Moffat (beta = 4.5) has
    # (r/alpha)^(2 - 2 beta) of its light beyond radius r, below 1e-7 at the
    # stamp's edge (r ~ 80, alpha ~ 7.5).
    from paper_1101_2254_gb300 import synth
    psf = synth.moffat_psf(11, 2.5).astype(np.float64)
    psf /= psf.sum()
    q, fwhm = 0.7, 6.0
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    d = oracle.make_desc(111, 111, 11, [oracle.GAUSSIAN], os_factor=8, os_box=40)
    img = oracle.render(d, np.array([55.2, 54.7, 2.0, fwhm, q, 35.0, 0.0]), psf)
    # the render covers the stamp; the PSF spills 5 px of light over the edge
    # only where the model is ~exp(-50^2/2 s^2), far below the tolerance
    assert abs(img.sum() - 2.0 * math.pi * q * 2.0 * s * s) < 1e-6 * img.sum()
    beta = 4.5
    al = fwhm * oracle.moffat_alpha_per_fwhm(beta)
    d = oracle.make_desc(161, 161, 11, [oracle.MOFFAT], os_factor=8, os_box=40)
    img = oracle.render(d, np.array([80.3, 80.6, 3.0, fwhm, beta, q, 110.0, 0.0]), psf)
    want = math.pi * q * 3.0 * al * al / (beta - 1.0)
    assert abs(img.sum() - want) < 2e-5 * want, (img.sum(), want)
