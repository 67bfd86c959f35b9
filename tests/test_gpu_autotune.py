"""The direct-convolution launch shape -- tile width (64 or 32), tile height
(32 or 16) and persistent grid (CTAs per SM) -- changes the work decomposition
only: models, chi^2 and Jacobian sums must be bit-identical under every shape,
and the tuner must leave a valid choice for every class it times."""
import numpy as np
import pytest

from paper_1101_2254_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_2254_gb300 import build, gf as gf_
    build.build()
    return gf_


SIZES = [(20, 20), (45, 70), (70, 150), (33, 97), (64, 64), (100, 37)]
P = 9


def case(gf):
    rng = np.random.default_rng(3)
    kinds = [synth.SERSIC, synth.SKY]
    params = [synth.random_params(kinds, rng, H, W) for H, W in SIZES]
    imgs = [rng.uniform(0.0, 2.0, H * W).astype(np.float32) for H, W in SIZES]
    sigs = [rng.uniform(0.5, 1.0, H * W).astype(np.float32) for H, W in SIZES]
    psfs = [synth.random_psf(P, 10 + i).ravel() for i in range(len(SIZES))]
    b = gf.make_batch([h for h, _ in SIZES], [w for _, w in SIZES], psf_size=P)
    d = gf.make_desc(1, 1, P, kinds, 3, 4, conv_method=gf.CONV_DIRECT)
    T = lambda xs: torch.as_tensor(np.concatenate(xs)).cuda()
    return d, b, np.array(params), T(imgs), T(sigs), T(psfs)


def run(gf, d, b, params, img, sig, psf):
    x2, m = gf.evaluate_batch(d, b, params, img, sig, psf, want_model=True)
    fixed = np.zeros(params.shape[1], np.uint8)
    fixed[7] = 1
    opts = gf.default_opts(max_iter=3)
    p, res = gf.lm_fit_batch(d, b, params, fixed, img, sig, psf, opts=opts)
    return x2.cpu().numpy(), m.cpu().numpy(), p, [r["chi2"] for r in res]


def test_tile_widths_give_identical_results(gf):
    d, b, params, img, sig, psf = case(gf)
    outs = []
    for tw in (64, 32):
        for _, W in SIZES:
            if ((W + 31) // 32) % 2 == 1:
                gf.set_conv_tile_width(P, W, tw)
        assert all(gf.conv_tile_width(P, W) == (tw if ((W + 31) // 32) % 2 else 64)
                   for _, W in SIZES)
        outs.append(run(gf, d, b, params, img, sig, psf))
    for a, c in zip(outs[0], outs[1]):
        assert np.array_equal(np.asarray(a), np.asarray(c))


def test_every_tile_height_and_grid_gives_identical_results(gf):
    d, b, params, img, sig, psf = case(gf)
    outs = []
    for th, cap in [(32, 8), (16, 8), (32, 4), (16, 16), (32, 1), (16, 2)]:
        gf.set_conv_tile_shape(P, th, cap)
        assert gf.conv_tile_shape(P, 64)[1:] == (th, cap)
        outs.append(run(gf, d, b, params, img, sig, psf))
    gf.set_conv_tile_shape(P, 32, 8)
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert np.array_equal(np.asarray(a), np.asarray(c))


def test_autotune_sets_a_width_per_odd_class(gf):
    d, b, params, img, sig, psf = case(gf)
    ref = run(gf, d, b, params, img, sig, psf)
    gf.autotune(d, b, psf)
    for _, W in SIZES:
        assert gf.conv_tile_width(P, W) in ((32, 64) if ((W + 31) // 32) % 2 else (64,))
        tw, th, cap = gf.conv_tile_shape(P, W)
        assert th in (16, 32) and cap in (4, 8, 16)
    after = run(gf, d, b, params, img, sig, psf)
    for a, c in zip(ref, after):
        assert np.array_equal(np.asarray(a), np.asarray(c))
