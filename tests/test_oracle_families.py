"""Pins of the oracle's further profile families (step 1 of the loop, Sec. 2):
the modified King profile, the Nuker law and unresolved point sources, each
against what its definition fixes independently of the oracle's own code --
closed-form total light by radial quadrature, values at its defining radii,
asymptotic slopes, identities with independently pinned families, the
cubic-convolution weights' known values and reproduction properties, and the
noiseless recovery of known parameters by the LM."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_1101_2254_gb300 import synth

KING, NUKER, PSF, MOFFAT, SERSIC, SKY = (oracle.KING, oracle.NUKER, oracle.PSF, oracle.MOFFAT,
                                         oracle.SERSIC, oracle.SKY)


def king(x0=3.0, y0=-2.0, I0=1.7, rc=2.5, rt=18.0, al=2.0, q=0.6, pa=35.0, c=0.0):
    return np.array([x0, y0, I0, rc, rt, al, q, pa, c])


def nuker(x0=1.0, y0=2.0, Ib=0.8, rb=5.0, al=2.0, be=4.0, ga=0.5, q=0.7, pa=120.0, c=0.0):
    return np.array([x0, y0, Ib, rb, al, be, ga, q, pa, c])


def along_major(kind, p, r):
    """The profile at distance r along the major axis (angle PA from +x)."""
    ipa = 7 if kind == KING else 8
    th = math.radians(p[ipa])
    return oracle.comp_value(kind, p, p[0] + r * math.cos(th), p[1] + r * math.sin(th))


def radial_flux(kind, p, rmax, q, points=None):
    """q * integral_0^rmax 2 pi r I(r) dr along the major axis (elliptical
    isophotes, c = 0: the area element of the ellipse family is q 2 pi r dr)."""
    v, _ = integrate.quad(lambda r: 2 * math.pi * r * along_major(kind, p, r), 0.0, rmax,
                          epsabs=0.0, epsrel=1e-11, limit=400, points=points)
    return q * v


# ------------------------------------------------------------------- King
def test_king_centre_and_truncation():
    p = king()
    assert abs(along_major(KING, p, 0.0) - p[2]) < 1e-14
    for r in (p[4], p[4] + 0.01, 2 * p[4]):
        assert along_major(KING, p, r) == 0.0
    assert along_major(KING, p, 0.999 * p[4]) > 0.0


@pytest.mark.parametrize("rc,rt", [(2.5, 18.0), (1.0, 40.0), (6.0, 9.0)])
def test_king_flux_closed_forms(rc, rt):
    # King (1962), alpha = 2: L = pi r_c^2 k [ln(1 + x_t^2) - 4 (1 - C) + 1 - C^2],
    # C = (1 + x_t^2)^(-1/2), k = I_0 / (1 - C)^2 (central value I_0)
    xt2 = (rt / rc) ** 2
    C = 1.0 / math.sqrt(1.0 + xt2)
    p = king(rc=rc, rt=rt, al=2.0, q=0.6)
    want = math.pi * rc * rc * p[2] / (1 - C) ** 2 * (math.log1p(xt2) - 4 * (1 - C) + 1 - C * C)
    assert abs(radial_flux(KING, p, rt, 0.6) - 0.6 * want) < 1e-9 * want
    # alpha = 1: I = I_0 (w - w_t) / (1 - w_t), w = 1 / (1 + x^2):
    # L = pi r_c^2 I_0 / (1 - w_t) [ln(1 + x_t^2) - x_t^2 / (1 + x_t^2)]
    wt = 1.0 / (1.0 + xt2)
    p = king(rc=rc, rt=rt, al=1.0, q=0.6)
    want = math.pi * rc * rc * p[2] / (1 - wt) * (math.log1p(xt2) - xt2 / (1 + xt2))
    assert abs(radial_flux(KING, p, rt, 0.6) - 0.6 * want) < 1e-9 * want


def test_king_pixel_sum_is_total_light():
    # a render (grid, oversampling everywhere, delta PSF) holds the closed-form light
    rc, rt = 2.0, 14.0
    p = np.concatenate([king(x0=20.3, y0=19.6, rc=rc, rt=rt, al=2.0, q=0.8, pa=20.0), [0.0]])
    xt2 = (rt / rc) ** 2
    C = 1.0 / math.sqrt(1.0 + xt2)
    want = 0.8 * math.pi * rc * rc * p[2] / (1 - C) ** 2 * (math.log1p(xt2) - 4 * (1 - C) + 1 - C * C)
    d = oracle.make_desc(40, 40, 1, [KING, SKY], 8, 40)
    img = oracle.render(d, p, np.ones((1, 1)))
    assert abs(img.sum() - want) < 2e-4 * want


# ------------------------------------------------------------------ Nuker
@pytest.mark.parametrize("al,be,ga", [(2.0, 4.0, 0.5), (1.0, 3.0, 0.0), (5.0, 2.5, 1.2)])
def test_nuker_break_value_and_slopes(al, be, ga):
    p = nuker(al=al, be=be, ga=ga)
    assert abs(along_major(NUKER, p, p[3]) - p[2]) < 1e-13 * p[2]
    # logarithmic slope -> -gamma inside the break and -beta far outside
    for r, slope in [(1e-4 * p[3], -ga), (1e4 * p[3], -be)]:
        h = 1e-4
        s = (math.log(along_major(NUKER, p, r * math.exp(h))) -
             math.log(along_major(NUKER, p, r * math.exp(-h)))) / (2 * h)
        assert abs(s - slope) < 2e-3 * max(1.0, abs(slope)), (r, s, slope)


@pytest.mark.parametrize("al,be,ga", [(2.0, 4.0, 0.5), (1.5, 5.0, 1.0), (3.0, 3.5, 0.2)])
def test_nuker_flux_beta_function(al, be, ga):
    # integral_0^inf 2 pi r I dr = 2 pi r_b^2 I_b 2^((beta-gamma)/alpha)
    #                              B((2 - gamma)/alpha, (beta - 2)/alpha) / alpha
    p = nuker(al=al, be=be, ga=ga, q=0.7)
    rb = p[3]
    want = 2 * math.pi * rb * rb * p[2] * 2 ** ((be - ga) / al) * special.beta(
        (2 - ga) / al, (be - 2) / al) / al
    # the inner region by quadrature, the far tail beyond R by its exact
    # integral in t (substitute u = t^-alpha: the tail is an incomplete beta)
    R = 50.0
    inner = radial_flux(NUKER, p, R * rb, 0.7, points=[rb])
    a_, b_ = (be - 2) / al, (2 - ga) / al
    x_ = 1.0 / (1.0 + R ** al)
    tail = 0.7 * 2 * math.pi * rb * rb * p[2] * 2 ** ((be - ga) / al) / al * special.betainc(
        a_, b_, x_) * special.beta(a_, b_)
    assert abs(inner + tail - 0.7 * want) < 1e-7 * want


def test_nuker_gamma0_alpha2_is_moffat():
    # gamma = 0, alpha = 2: I_b 2^(beta/2) (1 + (r/r_b)^2)^(-beta/2), a Moffat of
    # index beta/2 and scale alpha_M = r_b (its FWHM slot 2 r_b sqrt(2^(2/beta) - 1))
    be = 3.4
    p = nuker(al=2.0, be=be, ga=0.0)
    bm = be / 2
    fwhm = 2 * p[3] * math.sqrt(2 ** (1 / bm) - 1)
    pm = np.array([p[0], p[1], p[2] * 2 ** (be / 2), fwhm, bm, p[7], p[8], p[9]])
    rng = np.random.default_rng(3)
    for x, y in rng.uniform(-20, 20, (20, 2)):
        a, b = oracle.comp_value(NUKER, p, x, y), oracle.comp_value(MOFFAT, pm, x, y)
        assert abs(a - b) < 1e-12 * b


# ----------------------------------------------------------- point sources
def test_keys_weights_known_values():
    # Keys (1981), a = -1/2: the half-pixel weights are (-1/16, 9/16, 9/16, -1/16)
    for x, w in [(0.0, 1.0), (1.0, 0.0), (-1.0, 0.0), (2.0, 0.0), (0.5, 9 / 16),
                 (-1.5, -1 / 16), (1.5, -1 / 16), (3.7, 0.0)]:
        assert abs(oracle.keys_weight(x) - w) < 1e-15


def test_keys_partition_of_unity_and_linear_reproduction():
    rng = np.random.default_rng(5)
    for x in rng.uniform(-3.0, 3.0, 30):
        js = np.arange(math.floor(x) - 2, math.floor(x) + 4)
        w = np.array([oracle.keys_weight(j - x) for j in js])
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w * js).sum() - x) < 1e-13
        assert abs((w * js * js).sum() - x * x) < 1e-12  # quadratics too (a = -1/2)


def test_point_source_flux_centroid_and_integer_shift():
    H, W, P = 24, 30, 9
    psf = synth.moffat_psf(P, 3.0)
    for x0, y0 in [(11.3, 12.8), (14.0, 9.0), (7.61, 15.5)]:
        p = np.array([x0, y0, 37.5])
        d = oracle.make_desc(H, W, P, [PSF], 4, 8)  # an oversampled block at the centre
        ext = oracle.model_ext(d, p)
        c = (P - 1) // 2
        assert abs(ext.sum() - 37.5) < 1e-12
        ys, xs = np.mgrid[0:ext.shape[0], 0:ext.shape[1]]
        assert abs((ext * (xs - c)).sum() / ext.sum() - x0) < 1e-12
        assert abs((ext * (ys - c)).sum() / ext.sum() - y0) < 1e-12
        # the oversampled block leaves a point source as it is
        d1 = oracle.make_desc(H, W, P, [PSF], 1, 0)
        assert np.array_equal(ext, oracle.model_ext(d1, p))
        m = oracle.render(d, p, psf)
        if x0 == int(x0) and y0 == int(y0):
            want = np.zeros((H, W))
            i0, j0 = int(y0), int(x0)
            want[i0 - c:i0 + c + 1, j0 - c:j0 + c + 1] = 37.5 * psf.astype(np.float64)
            assert np.abs(m - want).max() < 1e-13


# ----------------------------------------------------------- fits
@pytest.mark.parametrize("kinds,params", [
    ([KING, SKY], [24.3, 22.8, 3.0, 3.0, 20.0, 2.2, 0.75, 40.0, 0.0, 0.05]),
    ([NUKER, SKY], [23.6, 24.2, 1.2, 4.0, 2.0, 3.5, 0.6, 0.8, 110.0, 0.0, 0.05]),
    ([SERSIC, PSF, SKY], [24.2, 23.9, 0.8, 5.0, 2.0, 0.7, 60.0, 0.0, 24.6, 23.3, 40.0, 0.05]),
])
def test_noiseless_recovery(kinds, params):
    H = W = 48
    P = 11
    psf = synth.moffat_psf(P, 3.0)
    p_true = np.array(params)
    d = oracle.make_desc(H, W, P, kinds, 4, 8)
    m = oracle.render(d, p_true, psf)
    sig = synth.noise_sigma(m)
    fixed = np.zeros(len(p_true), np.uint8)
    roles = synth.slot_roles(kinds)
    fixed[[i for i, r in enumerate(roles) if r == "c"]] = 1
    p0 = synth.perturb_guess(kinds, p_true, fixed, 1, frac=0.05)
    p, r = oracle.lm_fit(d, p0, fixed, psf, m, sig, opts=oracle.default_opts(ftol=1e-14, xtol=1e-14))
    free = fixed == 0
    rel = np.abs(p - p_true)[free] / np.maximum(np.abs(p_true[free]), 1.0)
    assert r["chi2"] < 1e-12 * m.size, r
    assert rel.max() < 1e-6, (rel, r)


# -------------------------------------------------------------- sky plane
SKYPLANE = oracle.SKYPLANE


def test_sky_plane_convolves_to_closed_form():
    # s0 + gx (x - x_c) + gy (y - y_c) through a (deliberately asymmetric) PSF:
    # sum(psf) (s0 + gx (j - x_c) + gy (i - y_c)) + gx M_x + gy M_y, with the
    # PSF's first moments M_x = sum psf[v][u] (c - u), M_y = sum psf[v][u] (c - v)
    H, W, P = 17, 23, 7
    c = (P - 1) // 2
    psf = synth.random_psf(P, 3).astype(np.float64)
    s0, gx, gy = 0.7, 0.013, -0.021
    d = oracle.make_desc(H, W, P, [SKYPLANE], 3, 4)
    m = oracle.render(d, np.array([s0, gx, gy]), psf)
    v, u = np.mgrid[0:P, 0:P]
    Ps, Mx, My = psf.sum(), (psf * (c - u)).sum(), (psf * (c - v)).sum()
    assert abs(Mx) > 1e-3 and abs(My) > 1e-3  # the test depends on the moments' sign
    i, j = np.mgrid[0:H, 0:W]
    xc, yc = (W - 1) / 2, (H - 1) / 2
    want = Ps * (s0 + gx * (j - xc) + gy * (i - yc)) + gx * Mx + gy * My
    assert np.abs(m - want).max() < 1e-13


def test_sky_plane_fit_is_linear_least_squares():
    # only the plane's three slots free: the LM ends at the weighted linear
    # least-squares solution over its three basis columns
    H, W, P = 40, 36, 9
    kinds = [SERSIC, SKYPLANE]
    p_true = np.array([18.2, 19.7, 3.0, 5.0, 2.0, 0.7, 40.0, 0.0, 0.4, 0.004, -0.003])
    psf = synth.moffat_psf(P, 3.0)
    d = oracle.make_desc(H, W, P, kinds, 4, 8)
    img, sig = synth.add_noise(oracle.render(d, p_true, psf), 5)
    fixed = np.ones(11, np.uint8)
    fixed[8:] = 0
    p0 = p_true.copy()
    p0[8:] = [0.0, 0.0, 0.0]
    p, r = oracle.lm_fit(d, p0, fixed, psf, img, sig,
                         opts=oracle.default_opts(ftol=1e-15, xtol=1e-15))
    # the closed form: columns = the convolved basis, target = image - galaxy
    gal = oracle.render(d, np.concatenate([p_true[:8], [0.0, 0.0, 0.0]]), psf)
    i, j = np.mgrid[0:H, 0:W]
    cols = [oracle.render(d, np.concatenate([p_true[:8], e]), psf) - gal
            for e in ([1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0])]
    A = np.stack([c.ravel() for c in cols], 1) / sig.ravel()[:, None]
    bvec = (img.astype(np.float64) - gal).ravel() / sig.ravel()
    want = np.linalg.lstsq(A, bvec, rcond=None)[0]
    assert np.abs(p[8:] - want).max() < 1e-9 * np.abs(want).max(), (p[8:], want)


def test_sky_plane_noiseless_recovery():
    H = W = 48
    P = 11
    kinds = [SERSIC, SKYPLANE]
    p_true = np.array([24.2, 23.9, 0.8, 5.0, 2.0, 0.7, 60.0, 0.0, 0.3, 0.002, -0.0015])
    psf = synth.moffat_psf(P, 3.0)
    d = oracle.make_desc(H, W, P, kinds, 4, 8)
    m = oracle.render(d, p_true, psf)
    sig = synth.noise_sigma(m)
    fixed = np.zeros(11, np.uint8)
    fixed[7] = 1
    p0 = synth.perturb_guess(kinds, p_true, fixed, 1, frac=0.05)
    p, r = oracle.lm_fit(d, p0, fixed, psf, m, sig, opts=oracle.default_opts(ftol=1e-14, xtol=1e-14))
    free = fixed == 0
    assert r["chi2"] < 1e-12 * m.size, r
    assert (np.abs(p - p_true)[free] / np.maximum(np.abs(p_true[free]), 1e-3)).max() < 1e-6


# ------------------------------------------------------- Fourier modes
SERSIC_F = oracle.SERSIC_F


def sersic_f(a=(0.0, 0.0, 0.0), phi=(0.0, 0.0, 0.0), n=1.0, q=0.7, pa=30.0):
    return np.array([0.0, 0.0, 1.0, 5.0, n, q, pa, 0.0, a[0], phi[0], a[1], phi[1], a[2], phi[2]])


def frame_point(p, rho, t):
    """(x, y) of circular radius rho and angle t in the component's frame
    (x' = rho cos t, y'/q = rho sin t)."""
    th = math.radians(p[6])
    xp, yp = rho * math.cos(t), p[5] * rho * math.sin(t)
    return p[0] + xp * math.cos(th) - yp * math.sin(th), p[1] + xp * math.sin(th) + yp * math.cos(th)


def test_fourier_zero_amplitudes_is_sersic():
    p = sersic_f(phi=(20.0, 50.0, 80.0), n=2.7)
    rng = np.random.default_rng(1)
    for x, y in rng.uniform(-15, 15, (20, 2)):
        a = oracle.comp_value(SERSIC_F, p, x, y)
        b = oracle.comp_value(SERSIC, p[:8], x, y)
        assert abs(a - b) <= 1e-14 * b


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_fourier_isophote_phase_and_amplitude(mode):
    # a single mode m of amplitude a and phase phi: along t = phi the radius is
    # scaled by (1 + a), along t = phi + 180/m degrees by (1 - a), so the
    # effective isophote (I = I_e) sits at rho = r_e / (1 +- a)
    m = (1, 3, 4)[mode]
    a, phi = 0.18, 35.0
    amps, phis = [0.0] * 3, [0.0] * 3
    amps[mode], phis[mode] = a, phi
    p = sersic_f(a=amps, phi=phis, n=2.0)
    for t_deg, g in [(phi, 1 + a), (phi + 180.0 / m, 1 - a)]:
        x, y = frame_point(p, p[3] / g, math.radians(t_deg))
        assert abs(oracle.comp_value(SERSIC_F, p, x, y) - p[2]) < 1e-12


@pytest.mark.parametrize("mode,a,phi", [(0, 0.2, 40.0), (1, -0.15, 10.0), (2, 0.25, -70.0)])
def test_fourier_single_mode_flux(mode, a, phi):
    # the radius r (1 + a cos m(t - phi)) rescales the light of each direction
    # by 1 / (1 + a cos ...)^2, whose mean over t is (1 - a^2)^(-3/2)
    from scipy import integrate
    amps, phis = [0.0] * 3, [0.0] * 3
    amps[mode], phis[mode] = a, phi
    p = sersic_f(a=amps, phi=phis, n=1.0)

    def f(rho, t):
        return oracle.comp_value(SERSIC_F, p, *frame_point(p, rho, t)) * rho

    v, _ = integrate.dblquad(f, 0.0, 2 * math.pi, 0.0, 150.0, epsabs=0.0, epsrel=1e-9)
    want = oracle.sersic_flux(1.0, 5.0, 1.0, 0.7) * (1 - a * a) ** -1.5
    assert abs(p[5] * v - want) < 1e-7 * want


def test_fourier_noiseless_recovery():
    H = W = 48
    P = 11
    kinds = [SERSIC_F, SKY]
    p_true = np.array([24.2, 23.9, 2.0, 6.0, 2.0, 0.75, 60.0, 0.0, 0.08, 30.0, 0.05, 10.0,
                       -0.06, 20.0, 0.3])
    psf = synth.moffat_psf(P, 3.0)
    d = oracle.make_desc(H, W, P, kinds, 4, 8)
    m = oracle.render(d, p_true, psf)
    sig = synth.noise_sigma(m)
    fixed = np.zeros(len(p_true), np.uint8)
    fixed[7] = 1
    p0 = synth.perturb_guess(kinds, p_true, fixed, 1, frac=0.03)
    p, r = oracle.lm_fit(d, p0, fixed, psf, m, sig, opts=oracle.default_opts(ftol=1e-14, xtol=1e-14))
    free = fixed == 0
    assert r["chi2"] < 1e-12 * m.size, r
    assert (np.abs(p - p_true)[free] / np.maximum(np.abs(p_true[free]), 1e-2)).max() < 1e-6
