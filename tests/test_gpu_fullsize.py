"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times, on sampled outputs the oracle computes one by one, and on
properties that hold at any size.

- 4096 uneven single-Sersic stamps (sides 32-256, Moffat 33x33) fitted in one
  batched LM call: every sampled stamp reaches the chi^2 of the oracle's fit
  from the same start under the same LM options (ftol = xtol = 1e-6).
- 64 stamps of 1024x1024 with a 255x255 PSF evaluated in one call by the
  tensor-core DFT path: sampled pixels against the oracle's direct sum, chi^2
  against the oracle's evaluation.
- 65536 64x64 stamps fitted from the learned start in one batched LM call: 512
  distinct oracle-rendered stamps, each repeated 128 times; every copy of a
  stamp must give the same fit bit for bit, and every sampled stamp reaches
  the chi^2 of the oracle's fit from the same start under the same options.
Every input is rendered by the oracle or drawn by the seeded generators; none
comes from the CUDA path."""
import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BENCH_TOL = 1e-6  # the benchmark's LM ftol and xtol
CHI2_REACH = 1e-4


@pytest.fixture(scope="module")
def gf():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_2254_gb300 import build, gf as gf_
    build.build()
    return gf_


def _render_one(job):
    """Oracle render plus seeded noise of one stamp (run in a spawned worker)."""
    H, W, P, kinds, osf, osb, params, psf, seed = job
    od = oracle.make_desc(H, W, P, kinds, osf, osb)
    return synth.add_noise(oracle.render(od, params, psf, method=1), seed)


def render_all(jobs):
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_render_one, jobs, chunksize=16))


def reach(od, p, psf, img, sig, x2_ref):
    x2 = oracle.evaluate(od, p, psf, img, sig, method=1)[0]
    return x2 <= x2_ref * (1 + CHI2_REACH)


def test_batch4096_full_size(gf):
    sts = synth.batch_stamps(4096)
    out = render_all([(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box, st.params, st.psf,
                       st.noise_seed) for st in sts])
    imgs = [im.ravel() for im, _ in out]
    sigs = [sg.ravel() for _, sg in out]
    descs = [oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box) for st in sts]
    s0 = sts[0]
    T = lambda xs: torch.as_tensor(np.concatenate(xs)).cuda()
    img_d, sig_d = T(imgs), T(sigs)
    psf_d = T([st.psf.ravel() for st in sts])
    p0 = np.array([st.guess() for st in sts])
    d = gf.make_desc(1, 1, s0.P, s0.kinds, s0.os_factor, 8)
    b = gf.make_batch([st.H for st in sts], [st.W for st in sts], psf_size=s0.P)
    opts = gf.default_opts(ftol=BENCH_TOL, xtol=BENCH_TOL)
    pg, res = gf.lm_fit_batch(d, b, p0, s0.fixed, img_d, sig_d, psf_d, opts=opts)
    status = np.array([r["status"] for r in res])
    assert np.all((status == gf.OK) | (status == gf.EMAXITER)), np.unique(status)
    assert (status == gf.OK).mean() > 0.95
    sample = np.random.default_rng(0).choice(4096, 12, replace=False)
    _, ro = oracle.lm_fit_batch([descs[i] for i in sample], p0[sample], s0.fixed,
                                np.concatenate([sts[i].psf.ravel() for i in sample]),
                                np.cumsum([0] + [sts[i].psf.size for i in sample[:-1]]),
                                np.concatenate([imgs[i] for i in sample]),
                                np.concatenate([sigs[i] for i in sample]),
                                np.cumsum([0] + [imgs[i].size for i in sample[:-1]]), method=1,
                                opts=oracle.default_opts(ftol=BENCH_TOL, xtol=BENCH_TOL))
    hits = [reach(descs[i], pg[i], sts[i].psf, imgs[i].reshape(sts[i].H, sts[i].W),
                  sigs[i].reshape(sts[i].H, sts[i].W), ro[k]["chi2"]) for k, i in enumerate(sample)]
    assert all(hits), hits


def test_precision64x1024_full_size(gf):
    n = 64
    sts = [synth.stamp512(seed=31 * 1000 + i, size=1024, psf_size=255) for i in range(n)]
    s0 = sts[0]
    P = s0.P
    rng = np.random.default_rng(3)
    img = (0.05 + 0.01 * rng.standard_normal((n, 1024, 1024))).astype(np.float32)
    sig = np.full((n, 1024, 1024), 0.01, np.float32)
    psf = np.stack([st.psf for st in sts])
    d = gf.make_desc(1024, 1024, P, s0.kinds, s0.os_factor, s0.os_box, conv_method=gf.CONV_DFT_TC)
    b = gf.make_batch([1024] * n, [1024] * n, psf_size=P)
    x2, m = gf.evaluate_batch(d, b, np.array([st.params for st in sts]), torch.as_tensor(img).cuda(),
                              torch.as_tensor(sig).cuda(), torch.as_tensor(psf).cuda(),
                              want_model=True)
    x2 = x2.cpu().numpy()
    m = m.view(n, 1024, 1024)
    floor = 5e-5  # the DFT path's absolute floor (its tests' DFT_FLOOR)
    for i in (0, 37, 63):
        st = sts[i]
        od = oracle.make_desc(1024, 1024, P, st.kinds, st.os_factor, st.os_box)
        ext = oracle.model_ext(od, st.params)
        flipped = st.psf.astype(np.float64)[::-1, ::-1]
        idx = np.random.default_rng(i).integers(0, 1024, (60, 2))
        want = np.array([np.sum(flipped * ext[y:y + P, x:x + P]) for y, x in idx])
        gm = m[i].cpu().numpy()
        got = gm[idx[:, 0], idx[:, 1]]
        assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + floor * gm.max()), i
        mo = oracle.convolve_fft(ext, st.psf.astype(np.float64))
        xo = oracle.chi2(img[i].astype(np.float64), sig[i].astype(np.float64), mo)
        assert abs(x2[i] - xo) <= 1e-4 * xo, (i, x2[i], xo)


def test_learned65536_full_size(gf):
    from paper_1101_2254_gb300 import learned
    from test_gpu_cnn import prior_params
    tr = learned.Trainer(seed=40, batch=512, lr=2e-4).train(2000)  # the benchmark's training
    nd, count = 512, 65536
    p = prior_params(nd, 7)
    fwhm = np.random.default_rng(8).uniform(2, 5, nd)
    psfs = np.stack([synth.moffat_psf(33, f, 3.0) for f in fwhm])
    od = oracle.make_desc(64, 64, 33, [oracle.SERSIC, oracle.SKY], 5, 8)
    out = render_all([(64, 64, 33, [oracle.SERSIC, oracle.SKY], 5, 8, p[i], psfs[i], 5000 + i)
                      for i in range(nd)])
    imgs = np.stack([im for im, _ in out])
    sigs = np.stack([sg for _, sg in out])
    rep = np.arange(count) % nd
    img = torch.as_tensor(imgs[rep]).cuda().reshape(-1)
    sig = torch.as_tensor(sigs[rep]).cuda().reshape(-1)
    psf = torch.as_tensor(psfs[rep]).cuda().reshape(-1)
    b = learned.uniform_batch(count)
    d = learned.stamp_desc()
    st, choice, _ = learned.starts(tr.w, b, img, sig, psf)
    st = st.cpu().numpy()
    fixed = np.zeros(9, np.uint8)
    fixed[7] = 1
    opts = gf.default_opts(ftol=BENCH_TOL, xtol=BENCH_TOL)
    pg, res = gf.lm_fit_batch(d, b, st, fixed, img, sig, psf, opts=opts)
    iters = np.array([r["iters"] for r in res])
    # every copy of a stamp starts and ends in the same place, bit for bit
    for k in range(nd):
        rows = np.nonzero(rep == k)[0]
        assert np.all(st[rows] == st[k]) and np.all(pg[rows] == pg[k]) and np.all(iters[rows] == iters[k])
    # sampled stamps reach the oracle's chi^2 from the same start
    sample = np.random.default_rng(1).choice(nd, 16, replace=False)
    _, ro = oracle.lm_fit_batch([od] * len(sample), st[sample], fixed, psfs[sample].ravel(),
                                np.arange(len(sample)) * 33 * 33, imgs[sample].ravel(),
                                sigs[sample].ravel(), np.arange(len(sample)) * 64 * 64, method=1,
                                opts=oracle.default_opts(ftol=BENCH_TOL, xtol=BENCH_TOL))
    hits = [reach(od, pg[i], psfs[i], imgs[i], sigs[i], ro[k]["chi2"]) for k, i in enumerate(sample)]
    assert all(hits), hits
