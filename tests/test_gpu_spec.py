"""GPU parity of the spectral-line path (the fitting loop in one dimension;
a cube is fitted spaxel by spaxel) against the FP64 oracle on the same seeded
inputs: models, chi^2, normal equations, and the batched LM fits."""
import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth

from gpu_util import CHI2_REL, assert_pix_close, param_bound_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1101_2254_gb300 import build, gf
    build.build()
    gf.lib()
    return gf


def f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def f64(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float64)).cuda()


def odesc(c: synth.SpecCube):
    return oracle.spec_desc(c.n_chan, c.n_lines, c.n_cont, np.shape(c.lsf)[-1])


def gdesc(gf, c: synth.SpecCube):
    return gf.make_spec_desc(c.n_chan, c.n_lines, c.n_cont, np.shape(c.lsf)[-1],
                             lsf_per_spectrum=np.ndim(c.lsf) == 2)


def lsf_of(c, b):
    return c.lsf[b] if np.ndim(c.lsf) == 2 else c.lsf


def render(c: synth.SpecCube, params=None):
    """Noise-free spectra by the oracle, then seeded noise (gain 1)."""
    params = c.params if params is None else params
    d = odesc(c)
    m = np.stack([oracle.spec_eval(d, params[b], lsf_of(c, b))[1] for b in range(c.count)])
    spec, sig = synth.add_noise(m, c.noise_seed)
    return m, spec, sig


# (count, n_chan, n_lines, n_cont, lsf_len, per-spectrum LSF): one channel; a
# ragged last chunk; the longest LSF; continuum only; lines only with the
# most lines; an LSF longer than the spectrum
MODEL_CASES = [(3, 1, 1, 1, 1, False), (4, 257, 2, 2, 9, False), (3, 700, 3, 3, 129, True),
               (2, 513, 0, 3, 25, False), (2, 100, 5, 0, 1, False), (2, 20, 1, 2, 129, False)]


@pytest.mark.parametrize("case", MODEL_CASES, ids=lambda c: "x".join(map(str, c[:5])))
def test_spec_model_parity(gf, case):
    count, N, K, nc, L, per = case
    c = synth.spec_batch(count, N, K, nc, L, seed=N + K, per_spectrum_lsf=per)
    g = gf.spec_model(gdesc(gf, c), c.params, f32(c.lsf)).cpu().numpy()
    d = odesc(c)
    for b in range(count):
        _, m = oracle.spec_eval(d, c.params[b], lsf_of(c, b))
        assert_pix_close(g[b], m, what=f"spec model {case} #{b}")


def test_spec_model_with_random_lsf_pins_the_flip(gf):
    c = synth.spec_batch(2, 300, 2, 1, 15, seed=5)
    c.lsf = synth.random_lsf(15, 9)
    g = gf.spec_model(gdesc(gf, c), c.params, f32(c.lsf)).cpu().numpy()
    for b in range(2):
        assert_pix_close(g[b], oracle.spec_eval(odesc(c), c.params[b], c.lsf)[1])


def test_spec_chi2_parity_with_invalid_channels(gf):
    c = synth.spec_batch(5, 611, 2, 2, 17, seed=3)
    _, spec, sig = render(c)
    spec[0, 3] = np.nan
    sig[1, 10] = 0.0
    sig[2, 20] = -1.0
    sig[3, 30] = np.inf
    p = c.guess()
    x2, m = gf.spec_eval(gdesc(gf, c), p, f32(spec), f32(sig), f32(c.lsf), want_model=True)
    x2 = x2.cpu().numpy()
    for b in range(c.count):
        xo, mo = oracle.spec_eval(odesc(c), p[b], c.lsf, spec[b], sig[b])
        assert abs(x2[b] - xo) <= CHI2_REL * xo, (b, x2[b], xo)
        assert_pix_close(m[b].cpu().numpy(), mo)


@pytest.mark.parametrize("analytic", [False, True])
def test_spec_normal_equations_parity(gf, analytic):
    c = synth.spec_batch(6, 480, 3, 2, 21, seed=11)
    _, spec, sig = render(c)
    p = c.guess()
    fixed = np.zeros(c.params.shape[1], np.uint8)
    fixed[1] = 1  # the continuum slope held
    r = gf.spec_normal(gdesc(gf, c), p, fixed, f32(spec), f32(sig), f32(c.lsf), analytic=analytic)
    A, g, x2 = (r[k].cpu().numpy() for k in ("A", "g", "chi2"))
    mode = oracle.JAC_ANALYTIC if analytic else oracle.JAC_FORWARD
    # FD columns difference two float32 models (5e-3, the stamps' bound); the
    # analytic columns carry float32 evaluation error only
    bound = 1e-4 if analytic else 5e-3
    for b in range(c.count):
        o = oracle.spec_jacobian(odesc(c), p[b], fixed, c.lsf, spec[b], sig[b], mode=mode)
        dA = np.abs(A[b] - o["A"]) / np.sqrt(np.outer(np.diag(o["A"]), np.diag(o["A"])))
        assert dA.max() < bound, (b, dA.max())
        gscale = np.sqrt(np.diag(o["A"]) * o["chi2"])
        assert np.all(np.abs(g[b] - o["g"]) <= bound * gscale), (b, g[b], o["g"])
        assert abs(x2[b] - o["chi2"]) <= CHI2_REL * o["chi2"]


def _fit_both(gf, c, spec, sig, start, analytic, fixed=None):
    opts = gf.default_opts(jac_mode=gf.JAC_ANALYTIC if analytic else gf.JAC_FD)
    pg, res = gf.spec_fit(gdesc(gf, c), start, fixed, f32(spec), f32(sig), f32(c.lsf), opts=opts)
    pg = pg.cpu().numpy()
    rg = gf.spec_results(res)
    oo = oracle.default_opts(jac_mode=oracle.JAC_ANALYTIC if analytic else oracle.JAC_FORWARD)
    po, ro = oracle.spec_fit_batch(odesc(c), start, fixed, c.lsf, spec, sig, opts=oo)
    return pg, rg, po, ro


@pytest.mark.parametrize("analytic", [False, True])
def test_spec_fit_reaches_the_oracle(gf, analytic):
    c = synth.spec_batch(24, 400, 3, 2, 21, seed=21)
    _, spec, sig = render(c)
    start = c.guess()
    pg, rg, po, ro = _fit_both(gf, c, spec, sig, start, analytic)
    d = odesc(c)
    for b in range(c.count):
        assert rg[b]["status"] in (gf.OK, gf.EMAXITER), (b, rg[b])
        assert ro[b]["status"] == oracle.CONVERGED, (b, ro[b])
        xg = oracle.spec_eval(d, pg[b], c.lsf, spec[b], sig[b])[0]
        assert xg <= ro[b]["chi2"] * (1 + CHI2_REL), (b, xg, ro[b]["chi2"])
        # the fitted parameters agree within 1e-3 relative (absolute for the
        # centres and widths, which are in channels), or within 1 % of the
        # parameter's statistical error where the chi^2 valley is that flat
        # (the stamps' rule)
        r = oracle.spec_jacobian(d, po[b], None, c.lsf, spec[b], sig[b],
                                 mode=oracle.JAC_ANALYTIC)
        sigma = np.sqrt(np.diag(np.linalg.inv(r["A"])))
        ok, dps, rel = param_bound_ok(pg[b], po[b], slice(None), sigma)
        assert ok, (b, rel.max(), dps.max(), pg[b], po[b])


def test_spec_fit_recovers_noiseless_parameters(gf):
    c = synth.spec_batch(8, 350, 2, 3, 15, seed=31)
    m, _, _ = render(c)
    sig = np.full_like(m, 1.0, dtype=np.float32)
    pg, rg, po, ro = _fit_both(gf, c, m.astype(np.float32), sig, c.guess(), analytic=True)
    rel = np.abs(pg - c.params) / np.maximum(np.abs(c.params), 1.0)
    assert rel.max() < 2e-4, rel.max()
    # at the float32 floor of a noiseless chi^2 the trials change it by
    # round-off only: the fit may end by the step test, crawl to max_iter or
    # see the damping grow to its cap; the parameters above are the check
    assert all(r["status"] in (gf.OK, gf.ENOCONV, gf.EMAXITER) for r in rg), rg


def test_spec_fit_is_independent_of_the_batch(gf):
    # a spectrum fitted alone and inside a batch gives the same bits
    c = synth.spec_batch(10, 333, 2, 2, 11, seed=41)
    _, spec, sig = render(c)
    start = c.guess()
    d = gdesc(gf, c)
    pb, rb = gf.spec_fit(d, start, None, f32(spec), f32(sig), f32(c.lsf))
    for b in (0, 7):
        ps, rs = gf.spec_fit(d, start[b:b + 1], None, f32(spec[b:b + 1]), f32(sig[b:b + 1]),
                             f32(c.lsf))
        assert torch.equal(ps[0], pb[b])
        assert gf.spec_results(rs)[0] == gf.spec_results(rb)[b]


def test_spec_per_spectrum_lsf(gf):
    c = synth.spec_batch(6, 256, 2, 1, 13, seed=51, per_spectrum_lsf=True)
    _, spec, sig = render(c)
    start = c.guess()
    pg, rg, po, ro = _fit_both(gf, c, spec, sig, start, analytic=False)
    d = odesc(c)
    for b in range(c.count):
        xg = oracle.spec_eval(d, pg[b], c.lsf[b], spec[b], sig[b])[0]
        assert xg <= ro[b]["chi2"] * (1 + CHI2_REL), (b, xg, ro[b]["chi2"])


def test_spec_fit_with_held_slots_and_bounds(gf):
    c = synth.spec_batch(6, 300, 2, 2, 9, seed=61)
    _, spec, sig = render(c)
    start = c.guess()
    fixed = np.zeros(8, np.uint8)
    fixed[[1, 7]] = 1  # slope and the second width held
    pg, rg, po, ro = _fit_both(gf, c, spec, sig, start, analytic=True, fixed=fixed)
    assert np.array_equal(pg[:, [1, 7]], start[:, [1, 7]])
    d = odesc(c)
    for b in range(c.count):
        xg = oracle.spec_eval(d, pg[b], c.lsf, spec[b], sig[b])[0]
        assert xg <= ro[b]["chi2"] * (1 + CHI2_REL)


def test_spec_fit_of_an_all_invalid_spectrum_stops(gf):
    # no valid channel: every slot is held, the first step is zero and the
    # fit stops as converged, like the oracle
    c = synth.spec_batch(2, 64, 1, 1, 5, seed=71)
    _, spec, sig = render(c)
    sig[1, :] = 0.0
    pg, rg, po, ro = _fit_both(gf, c, spec, sig, c.guess(), analytic=False)
    assert rg[1]["status"] == gf.OK and ro[1]["status"] == oracle.CONVERGED
    assert rg[1]["iters"] == ro[1]["iters"] == 1
    assert np.array_equal(pg[1], np.maximum(c.guess()[1], [-np.inf, -np.inf, -np.inf, 0.25]))


def test_spec_cube_full_size_sampled(gf):
    # the benchmark's cube (128 x 128 spaxels, 2048 channels) in its launch
    # configuration; the oracle refits 6 sampled spaxels from the same start
    c = synth.spec_cube(128, 2048, seed=0)
    d = gdesc(gf, c)
    _, spec_h, sig_h = render(c)  # rendered by the oracle
    start = c.guess()
    pg, res = gf.spec_fit(d, start, None, f32(spec_h), f32(sig_h), f32(c.lsf))
    pg = pg.cpu().numpy()
    rg = gf.spec_results(res)
    ok = sum(r["status"] == gf.OK for r in rg)
    assert ok >= 0.99 * c.count, ok
    od = odesc(c)
    for b in np.random.default_rng(0).choice(c.count, 6, replace=False):
        po, ro = oracle.spec_fit(od, start[b], None, c.lsf, spec_h[b], sig_h[b])
        xg = oracle.spec_eval(od, pg[b], c.lsf, spec_h[b], sig_h[b])[0]
        assert xg <= ro["chi2"] * (1 + CHI2_REL), (b, xg, ro["chi2"])
