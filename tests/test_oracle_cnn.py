"""Pins of the oracle's initial-guess network (forward conventions, analytic
gradient) and of its moments-based default guess."""
import math

import numpy as np
import pytest

import oracle

LAYERS = [(1, 32, 64, True), (32, 64, 32, True), (64, 64, 16, True), (64, 128, 8, True),
          (2048, 32, 1, False), (32, 8, 1, False)]


def he_init(seed):
    rng = np.random.default_rng(seed)
    w = []
    for cin, cout, _, conv in LAYERS:
        fan = cin * (9 if conv else 1)
        w.append(rng.standard_normal(cout * fan) * math.sqrt(2.0 / fan))
        w.append(rng.uniform(-0.1, 0.1, cout))
    return np.concatenate(w)


def numpy_forward(w, x):
    """Independent forward with scipy's 2-D correlation, stride-2 subsampling."""
    from scipy.signal import correlate2d
    off = 0
    a = x[None]  # (c, h, w)
    outs = None
    for li, (cin, cout, hin, conv) in enumerate(LAYERS):
        if conv:
            W = w[off:off + cout * cin * 9].reshape(cout, cin, 3, 3)
            off += cout * cin * 9
            b = w[off:off + cout]
            off += cout
            pad = np.pad(a, ((0, 0), (1, 1), (1, 1)))
            out = np.zeros((cout, hin // 2, hin // 2))
            for co in range(cout):
                acc = np.zeros((hin, hin))
                for ci in range(cin):
                    acc += correlate2d(pad[ci], W[co, ci], mode="valid")
                out[co] = acc[::2, ::2] + b[co]
            a = np.maximum(out, 0.0)
        else:
            W = w[off:off + cout * cin].reshape(cout, cin)
            off += cout * cin
            b = w[off:off + cout]
            off += cout
            z = W @ a.reshape(-1) + b
            a = z if li == 5 else np.maximum(z, 0.0)
    return a


def test_parameter_count():
    assert oracle.cnn_nparams() == 195432


def test_forward_matches_independent_correlation():
    w = he_init(1)
    x = np.random.default_rng(2).standard_normal((2, 64, 64))
    y = oracle.cnn_forward(w, x)
    for s in range(2):
        want = numpy_forward(w, x[s])
        assert np.abs(y[s] - want).max() < 1e-10 * max(1.0, np.abs(want).max())


def test_gradient_matches_central_differences():
    w = he_init(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 64, 64))
    t = rng.standard_normal((2, 8))
    loss, g = oracle.cnn_loss_grad(w, x, t)
    # a spread of parameters from every layer, weights and biases
    idx = np.unique(np.concatenate([rng.integers(0, w.size, 40), [0, 320, 18816, 55744, 129600,
                                                                 195168, w.size - 1]]))
    h = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        fd = (oracle.cnn_loss_grad(wp, x, t)[0] - oracle.cnn_loss_grad(wm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max() + 1e-7 * abs(g[i]), (i, fd, g[i])
    # the loss is the mean squared error of the forward outputs
    y = oracle.cnn_forward(w, x)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-12 * loss


def test_default_guess_on_a_sampled_gaussian():
    # sky + elliptical Gaussian: first and second moments give the centre, axis
    # ratio and angle exactly; the median border pixel gives the sky
    H = W = 96
    x0, y0, sx, sy, pa, sky = 47.3, 45.8, 6.0, 3.6, 35.0, 0.05
    th = math.radians(pa)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    dx, dy = xx - x0, yy - y0
    xp = dx * math.cos(th) + dy * math.sin(th)
    yp = -dx * math.sin(th) + dy * math.cos(th)
    img = sky + 10.0 * np.exp(-0.5 * (xp ** 2 / sx ** 2 + yp ** 2 / sy ** 2))
    g = oracle.default_guess(img)
    assert abs(g[8] - sky) < 1e-9
    assert abs(g[0] - x0) < 1e-6 and abs(g[1] - y0) < 1e-6
    assert abs(g[5] - sy / sx) < 1e-4
    assert abs(g[6] - pa) < 1e-3
    # half-light semi-major axis of a Gaussian: sx sqrt(2 ln 2), to the 0.25 px grid
    assert abs(g[3] - sx * math.sqrt(2 * math.log(2))) <= 0.26
    assert g[4] == 2.0 and g[7] == 0.0
    # I_e reproduces the summed flux through the closed form
    F = (img - sky)[img - sky > 0].sum()
    assert abs(oracle.sersic_flux(g[2], g[3], 2.0, g[5]) - F) < 1e-9 * F
