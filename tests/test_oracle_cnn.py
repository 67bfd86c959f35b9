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


def test_input_scaling_median_ring_and_asinh():
    # ring sigmas are a permutation of 1..252: the median is (126 + 127) / 2
    rng = np.random.default_rng(5)
    H = W = 64
    sig = rng.uniform(300.0, 400.0, (H, W))
    ring = np.zeros((H, W), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    sig[ring] = rng.permutation(np.arange(1.0, 253.0))
    z = rng.standard_normal((H, W)) * 3.0
    img = 126.5 * np.sinh(z)
    x = oracle.cnn_input(img, sig)
    assert np.abs(x - z).max() < 1e-12 * np.abs(z).max()


def test_target_encoding_reference_points_and_round_trip():
    # the centre of every scaled range encodes to zero
    n = 3.25
    q = 0.6
    re = math.sqrt(80.0)
    F = 10.0 ** 3.5
    ie = F / oracle.sersic_flux(1.0, re, n, q)
    t = oracle.cnn_encode([31.5, 31.5, ie, re, n, q, 45.0], 64, 64)
    assert np.abs(t[:6]).max() < 1e-12
    assert abs(t[6]) < 1e-15 and abs(t[7] - 1.0) < 1e-15  # 2 * 45 deg = 90 deg
    # range ends: r_e = 40 and F = 1e5 map to +1, n = 0.5 and q = 0.2 to -1
    ie = 1e5 / oracle.sersic_flux(1.0, 40.0, 0.5, 0.2)
    t = oracle.cnn_encode([30.5, 32.0, ie, 40.0, 0.5, 0.2, 135.0], 64, 64)
    assert np.allclose(t, [-1.0, 0.5, 1.0, 1.0, -1.0, -1.0, 0.0, -1.0], atol=1e-12)
    # decode inverts encode over the training prior
    rng = np.random.default_rng(6)
    for _ in range(50):
        p = np.array([31.5 + rng.uniform(-1, 1), 31.5 + rng.uniform(-1, 1), 0.0,
                      math.exp(rng.uniform(math.log(2), math.log(40))), rng.uniform(0.5, 6),
                      rng.uniform(0.2, 1.0), rng.uniform(0, 180), 0.0])
        p[2] = math.exp(rng.uniform(math.log(1e2), math.log(1e5))) / oracle.sersic_flux(
            1.0, p[3], p[4], p[5])
        back = oracle.cnn_decode(oracle.cnn_encode(p, 64, 64), 64, 64)
        assert np.abs(back[[0, 1, 4, 5]] - p[[0, 1, 4, 5]]).max() < 1e-12
        assert abs(back[2] / p[2] - 1) < 1e-12 and abs(back[3] / p[3] - 1) < 1e-12
        dpa = (back[6] - p[6] + 90.0) % 180.0 - 90.0
        assert abs(dpa) < 1e-9 and back[7] == 0.0
    # outside the flux domain the amplitude is not a number
    assert math.isnan(oracle.cnn_decode([0, 0, 0, 0, 4.0, 0, 1, 0], 64, 64)[2])


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000),
                        # ties: exactly half-way between two bfloat16 neighbours
                        (1.0 + (2 * np.arange(1, 200) + 1) * 2.0 ** -8) * 0.75,
                        [0.0, -0.0, 1.0, -2.5, 3.0e38, 1e-40]]).astype(np.float32)
    want = torch.as_tensor(v).bfloat16().float().numpy().astype(np.float64)
    got = np.array([oracle.bf16_round(float(a)) for a in v])
    assert np.array_equal(got, want)


def test_bf16_activation_mode():
    w = he_init(12)
    rng = np.random.default_rng(13)
    x = rng.standard_normal((2, 64, 64))
    t = rng.standard_normal((2, 8))
    y0 = oracle.cnn_forward(w, x)
    y1 = oracle.cnn_forward(w, x, bf16_act=True)
    # 8-bit activations perturb the outputs at the 2^-9 level, not more
    assert not np.array_equal(y0, y1)
    assert np.abs(y1 - y0).max() <= 2e-2 * np.abs(y0).max()
    # the rounded conv outputs do not depend on the fully connected layers, so
    # the gradient there is the exact derivative: central differences agree
    loss, g = oracle.cnn_loss_grad(w, x, t, bf16_act=True)
    assert abs(loss - np.mean((y1 - t) ** 2)) < 1e-12 * loss
    h = 1e-6
    for i in list(rng.integers(129600, 195432, 12)) + [195424, 195431]:
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        fd = (oracle.cnn_loss_grad(wp, x, t, True)[0] - oracle.cnn_loss_grad(wm, x, t, True)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * np.abs(g).max(), (i, fd, g[i])
